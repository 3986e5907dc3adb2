// count_flops.cpp -- algorithmic FP64 operation counts of the update, per cell,
// measured on the oracle's own formulas.  MEASUREMENT INFRASTRUCTURE ONLY (it
// never feeds the CUDA path): the oracle source is compiled as C++ with every
// double replaced by a counting number type, each oracle function is applied
// to the states of a seeded workload, and the counts of one call are combined
// into the minimal per-cell work of each stage (each face flux once, each cell
// reconstructed once per direction, each cell converted once per stage).
//
// Flop convention: add, subtract, multiply, divide and square root count one
// each; comparisons, min/max and fabs are counted separately (they occupy the
// FP64 pipe on GB300 but are not floating-point arithmetic).
//
// Build and run: g++ -O1 -std=c++17 -o /tmp/count_flops oracle/count_flops.cpp
//                /tmp/count_flops 24
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

struct Tally { double add = 0, mul = 0, div = 0, sqrt_ = 0, cmp = 0; };
static Tally g_t;

struct Num {
  double v;
  Num() = default;
  Num(double x) : v(x) {}
  explicit operator double() const { return v; }
  explicit operator int() const { return (int)v; }
};
static inline Num operator+(Num a, Num b) { g_t.add++; return Num(a.v + b.v); }
static inline Num operator-(Num a, Num b) { g_t.add++; return Num(a.v - b.v); }
static inline Num operator*(Num a, Num b) { g_t.mul++; return Num(a.v * b.v); }
static inline Num operator/(Num a, Num b) { g_t.div++; return Num(a.v / b.v); }
static inline Num operator-(Num a) { return Num(-a.v); }
static inline Num &operator+=(Num &a, Num b) { a = a + b; return a; }
static inline Num &operator-=(Num &a, Num b) { a = a - b; return a; }
static inline bool operator<(Num a, Num b) { g_t.cmp++; return a.v < b.v; }
static inline bool operator>(Num a, Num b) { g_t.cmp++; return a.v > b.v; }
static inline bool operator<=(Num a, Num b) { g_t.cmp++; return a.v <= b.v; }
static inline bool operator>=(Num a, Num b) { g_t.cmp++; return a.v >= b.v; }
static inline bool operator==(Num a, Num b) { g_t.cmp++; return a.v == b.v; }
static inline bool operator!=(Num a, Num b) { g_t.cmp++; return a.v != b.v; }
static inline bool operator!(Num a) { g_t.cmp++; return !a.v; }
static inline Num sqrt(Num a) { g_t.sqrt_++; return Num(std::sqrt(a.v)); }
static inline Num fabs(Num a) { return Num(std::fabs(a.v)); }
static inline Num ceil(Num a) { return Num(std::ceil(a.v)); }

#define double Num
#include "qk_oracle.c"
#undef double

static double flops(const Tally &t) { return t.add + t.mul + t.div + t.sqrt_; }
static Tally diff(const Tally &a, const Tally &b) {
  Tally d;
  d.add = a.add - b.add; d.mul = a.mul - b.mul; d.div = a.div - b.div;
  d.sqrt_ = a.sqrt_ - b.sqrt_; d.cmp = a.cmp - b.cmp;
  return d;
}
static void print(const char *name, Tally t, double n) {
  std::printf("  \"%s\": {\"flops\": %.1f, \"add\": %.1f, \"mul\": %.1f, \"div\": %.2f, "
              "\"sqrt\": %.2f, \"cmp\": %.1f}", name, flops(t) / n, t.add / n, t.mul / n,
              t.div / n, t.sqrt_ / n, t.cmp / n);
}

// seeded smooth random states (the statistics of the limiter and Riemann-solver
// branches follow the workload: lognormal density, T_r ~ U(0.5, 2))
static double urand(uint64_t &s) {
  s = s * 6364136223846793005ull + 1442695040888963407ull;
  return ((s >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

int main(int argc, char **argv) {
  const int n = argc > 1 ? std::atoi(argv[1]) : 24;
  const int ng = 4, sx = n + 2 * ng;
  const int64_t len = (int64_t)sx * sx * sx;
  int32_t lo[3] = {0, 0, 0}, nn[3] = {n, n, n}, dom[3] = {n, n, n};
  int64_t off = 0;
  or_grid *g = or_grid_create(1, lo, nn, &off, dom, ng);
  std::vector<Num> f[9];
  for (auto &v : f) v.assign(len, Num(0.0));
  uint64_t seed = 2110;
  const double gam = 5.0 / 3.0, cv = 1.0 / (gam - 1.0), c = 100.0, chat = 10.0 * std::sqrt(gam);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        int64_t e = ((int64_t)(k + ng) * sx + (j + ng)) * sx + (i + ng);
        double x = 2 * M_PI * (i + 0.5) / n, y = 2 * M_PI * (j + 0.5) / n, z = 2 * M_PI * (k + 0.5) / n;
        double rho = std::exp(0.8 * std::sin(x + 2 * y) * std::cos(z) + 0.2 * (urand(seed) - 0.5));
        double vx = 0.3 * std::sin(y + z), vy = 0.3 * std::cos(x), vz = 0.2 * std::sin(x + y);
        double Tg = 1.0 + 0.3 * urand(seed), Tr = 0.5 + 1.5 * urand(seed);
        double Er = Tr * Tr * Tr * Tr, fr = 0.5 * urand(seed);
        f[0][e] = rho; f[1][e] = rho * vx; f[2][e] = rho * vy; f[3][e] = rho * vz;
        f[4][e] = rho * cv * Tg + 0.5 * rho * (vx * vx + vy * vy + vz * vz);
        f[5][e] = Er; f[6][e] = c * Er * fr; f[7][e] = -0.5 * c * Er * fr; f[8][e] = 0.3 * c * Er * fr;
      }
  or_params p;
  std::memset(&p, 0, sizeof(p));
  p.gamma = gam; p.cfl = 0.3; p.a_r = 1.0; p.c = c; p.chat = chat; p.c_v = cv;
  p.kappa_P = 1.0; p.kappa_R = 1.0; p.eps_newton = 1e-10;
  p.dx[0] = p.dx[1] = p.dx[2] = 1.0 / n;
  p.max_iter = 400; p.nsub_max = 10; p.tau_correction = 1;
  Num *U[5], *R[4];
  for (int q = 0; q < 5; ++q) U[q] = f[q].data();
  for (int q = 0; q < 4; ++q) R[q] = f[5 + q].data();
  const double ncell = (double)n * n * n;

  // --- per-function counts, averaged over every cell / face of the workload
  Tally t0 = g_t;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        int64_t e = cell_index(g, 0, i, j, k);
        Num Uc[5], q[5];
        for (int v = 0; v < 5; ++v) Uc[v] = U[v][e];
        con2prim(Uc, p.gamma, q);
      }
  Tally c2p = diff(g_t, t0);
  // PPM: once per cell, direction and primitive; HLLC: once per face
  Tally ppm_t, hllc_t, rppm_t, rface_t;
  double nppm = 0, nface = 0;
  for (int d = 0; d < 3; ++d)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int c3[3] = {i, j, k};
          Num w[5][6], wL[5], wR[5], dum, F[5];
          gather_prims(g, &p, U, 0, c3, d, -2, w);  // cells c-2 .. c+3
          Tally a = g_t;
          for (int v = 0; v < 5; ++v) or_ppm_cell(&w[v][0], &dum, &wL[v]);
          Tally b = g_t;
          for (int v = 0; v < 5; ++v) or_ppm_cell(&w[v][1], &wR[v], &dum);
          Tally cc = g_t;
          or_hllc(wL, wR, d, p.gamma, F);  // (no flattening in the benchmark workloads)
          Tally dd = g_t;
          Tally x = diff(b, a);
          ppm_t.add += x.add; ppm_t.mul += x.mul; ppm_t.div += x.div; ppm_t.sqrt_ += x.sqrt_; ppm_t.cmp += x.cmp;
          (void)cc;
          Tally h = diff(dd, cc);
          hllc_t.add += h.add; hllc_t.mul += h.mul; hllc_t.div += h.div; hllc_t.sqrt_ += h.sqrt_; hllc_t.cmp += h.cmp;
          nppm += 5; nface += 1;
          // radiation: 4 reconstructions, then the face flux minus its own
          // reconstructions (closures of both states, wavespeed closures, HLL)
          Num r[4][6], rL[4], rR[4], rd;
          gather_rad(g, &p, R, 0, c3, d, -2, r);
          Tally ra = g_t;
          for (int v = 0; v < 4; ++v) or_ppm_cell(&r[v][0], &rd, &rL[v]);
          Tally rb = g_t;
          Tally y = diff(rb, ra);
          rppm_t.add += y.add; rppm_t.mul += y.mul; rppm_t.div += y.div; rppm_t.sqrt_ += y.sqrt_; rppm_t.cmp += y.cmp;
          Num Fo[4];
          Tally fa = g_t;
          rad_face_flux(g, &p, R, U[0], 0, c3, d, -2, Fo);
          Tally fb = g_t;
          Tally z = diff(fb, fa);  // includes 8 reconstructions and 6-cell gather
          rface_t.add += z.add; rface_t.mul += z.mul; rface_t.div += z.div; rface_t.sqrt_ += z.sqrt_; rface_t.cmp += z.cmp;
        }
  // gather_rad inside rad_face_flux: 6 cells x 3 divisions; 8 ppm calls
  Tally gat0 = g_t;
  {
    int c3[3] = {n / 2, n / 2, n / 2};
    Num r[4][6];
    gather_rad(g, &p, R, 0, c3, 0, -2, r);
  }
  Tally gat = diff(g_t, gat0);
  // exchange: one call per cell
  Tally ex0 = g_t;
  std::vector<Num> Ucopy[5], Rcopy[4];
  for (int q = 0; q < 5; ++q) Ucopy[q] = f[q];
  for (int q = 0; q < 4; ++q) Rcopy[q] = f[5 + q];
  Num *Uc[5], *Rc[4];
  for (int q = 0; q < 5; ++q) Uc[q] = Ucopy[q].data();
  for (int q = 0; q < 4; ++q) Rc[q] = Rcopy[q].data();
  int64_t info[4];
  double dtr = 0.3 * (1.0 / n) / chat;
  or_exchange(g, &p, Uc, Rc, dtr, 0, nullptr, nullptr, info);
  Tally exch = diff(g_t, ex0);

  std::printf("{\n  \"cells\": %d,\n  \"convention\": \"add+sub+mul+div+sqrt, per unit\",\n", n * n * n);
  print("con2prim_per_cell", c2p, ncell); std::printf(",\n");
  print("ppm_per_call", ppm_t, nppm); std::printf(",\n");
  print("hllc_per_face", hllc_t, nface); std::printf(",\n");
  print("rad_ppm_per_call", rppm_t, 4 * nface); std::printf(",\n");
  print("rad_face_flux_incl_8ppm_and_gather", rface_t, nface); std::printf(",\n");
  print("rad_gather_6cells", gat, 1.0); std::printf(",\n");
  print("exchange_per_cell", exch, ncell); std::printf(",\n");
  std::printf("  \"newton_mean_iterations\": %.3f\n}\n", (double)info[3] / ncell);
  or_grid_destroy(g);
  return 0;
}
