// qk_noalloc.cu -- conservation sums for callers that must not allocate GPU
// memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// conservation totals: a diagnostics hook that runs between steps under a
// strict memory budget, code under an external memory manager that owns every
// device allocation of the process, or a caller that has not (and will not)
// create a qk context.  qk_conserved_sums_noalloc serves them.  (It launches
// kernels and synchronises its stream, so it must not be called from a CUDA
// stream host callback, where CUDA API calls are not allowed.)  It takes the
// patch table and the fields directly and keeps all of its working memory in
// one fixed-size array in the library's device memory (a file-scope
// __device__ array, so every GPU that loads the library holds it until the
// process exits).  It computes the same sums, with the same kernels and the
// same fixed reduction order, as qk_conserved_sums.
#include <cstdio>
#include <mutex>

#include "qk_internal.cuh"

namespace qk {

// Layout of the static scratch (bytes):
//   patch table copy     QK_NOALLOC_MAX_BOXES x sizeof(qk_box)
//   device patch table   QK_NOALLOC_MAX_BOXES x sizeof(DevBox)
//   interior-cell prefix (QK_NOALLOC_MAX_BOXES + 1) x 8
//   per-block partials   kMaxBlocks x QK_NSUMS x 2 x 8
//   result               QK_NSUMS x 8
constexpr int kMaxBlocks = 1024;
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffBoxIn = 0;
constexpr size_t kOffDevBox = align256(kOffBoxIn + sizeof(qk_box) * QK_NOALLOC_MAX_BOXES);
constexpr size_t kOffPrefix = align256(kOffDevBox + sizeof(DevBox) * QK_NOALLOC_MAX_BOXES);
constexpr size_t kOffPartials = align256(kOffPrefix + 8 * (QK_NOALLOC_MAX_BOXES + 1));
constexpr size_t kOffOut = align256(kOffPartials + 8 * 2 * QK_NSUMS * kMaxBlocks);
constexpr size_t kScratchBytes = align256(kOffOut + 8 * QK_NSUMS);
static_assert(kScratchBytes <= QK_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds its stated size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[QK_NOALLOC_SCRATCH_BYTES];

// Build the device patch table and the interior-cell prefix from the copied
// qk_box array (one thread: at most QK_NOALLOC_MAX_BOXES patches).
__global__ void noalloc_table_kernel(unsigned char *base, int nbox, int ng) {
  const qk_box *in = reinterpret_cast<const qk_box *>(base + kOffBoxIn);
  DevBox *db = reinterpret_cast<DevBox *>(base + kOffDevBox);
  long long *cell0 = reinterpret_cast<long long *>(base + kOffPrefix);
  long long acc = 0;
  for (int b = 0; b < nbox; ++b) {
    const qk_box q = in[b];
    DevBox d;
    for (int a = 0; a < 3; ++a) {
      d.lo[a] = q.lo[a];
      d.n[a] = q.n[a];
    }
    d.sx = q.n[0] + 2 * ng;
    d.sy = q.n[1] + 2 * ng;
    d.off = q.offset;
    d.cell0 = acc;
    db[b] = d;
    cell0[b] = acc;
    acc += (long long)q.n[0] * q.n[1] * q.n[2];
  }
  cell0[nbox] = acc;
}

// Device address of the scratch array, looked up once per device (with that
// device current) and kept for the life of the process.  A cudaDeviceReset
// unloads the module, so the kept address does not survive it (documented in
// the header).
static unsigned char *scratch_address(int dev, cudaError_t *err) {
  static std::mutex mu;
  static unsigned char *addr[64] = {};
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  if (!addr[dev]) {
    void *p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    addr[dev] = static_cast<unsigned char *>(p);
  }
  *err = cudaSuccess;
  return addr[dev];
}

}  // namespace qk

using namespace qk;

// Write a message into the caller's buffer (no allocation).
static void report(char *err, int32_t errlen, const char *fmt, int a = 0, int b = 0) {
  if (err && errlen > 0) snprintf(err, (size_t)errlen, fmt, a, b, b);
}

extern "C" int qk_conserved_sums_noalloc(const qk_params *p, const qk_box *boxes, int32_t nbox,
                                         int32_t nghost, int32_t precision, int64_t field_len,
                                         void *const hydro[5], void *const rad[4],
                                         double out[QK_NSUMS], void *stream, char *err,
                                         int32_t errlen) {
  if (err && errlen > 0) err[0] = 0;
  if (!p || !boxes || !hydro || !out) {
    report(err, errlen, "qk_conserved_sums_noalloc: params, boxes, hydro and out must be non-NULL");
    return QK_EINVAL;
  }
  if (nbox < 1 || nbox > QK_NOALLOC_MAX_BOXES) {
    report(err, errlen,
           "qk_conserved_sums_noalloc: %d patches; this entry point takes 1 to %d "
           "(its fixed scratch holds at most %d patches)",
           (int)nbox, QK_NOALLOC_MAX_BOXES);
    return QK_EINVAL;
  }
  if (nghost < 0 || nghost > 16 || (precision != QK_FP64 && precision != QK_FP32_MIXED)) {
    report(err, errlen, "qk_conserved_sums_noalloc: nghost must be in [0, 16] and precision "
                        "QK_FP64 or QK_FP32_MIXED");
    return QK_EINVAL;
  }
  for (int q = 0; q < 5; ++q)
    if (!hydro[q]) {
      report(err, errlen, "qk_conserved_sums_noalloc: a hydro field pointer is NULL");
      return QK_EINVAL;
    }
  if (rad)
    for (int q = 0; q < 4; ++q)
      if (!rad[q]) {
        report(err, errlen, "qk_conserved_sums_noalloc: a radiation field pointer is NULL");
        return QK_EINVAL;
      }
  long long ncells = 0;
  for (int b = 0; b < nbox; ++b) {
    const qk_box &q = boxes[b];
    if (q.n[0] < 1 || q.n[1] < 1 || q.n[2] < 1 || q.offset < 0) {
      report(err, errlen, "qk_conserved_sums_noalloc: patch %d has an empty extent or a "
                          "negative offset", b);
      return QK_EINVAL;
    }
    // the padded patch must lie inside every field array (no read past them)
    const long long sx = (long long)q.n[0] + 2 * nghost, sy = (long long)q.n[1] + 2 * nghost,
                    sz = (long long)q.n[2] + 2 * nghost;
    if (q.n[0] > (1 << 20) || q.n[1] > (1 << 20) || q.n[2] > (1 << 20) ||
        q.offset > field_len || sx * sy * sz > field_len - q.offset) {
      report(err, errlen, "qk_conserved_sums_noalloc: patch %d with its ghost cells ends "
                          "beyond field_len", b);
      return QK_EINVAL;
    }
    ncells += (long long)q.n[0] * q.n[1] * q.n[2];
  }
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  unsigned char *base = e == cudaSuccess ? scratch_address(dev, &e) : nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  // the same block count as qk_conserved_sums gives the same reduction order
  const int nblocks = nsm * 2 < 1 ? 1 : nsm * 2;
  if (e == cudaSuccess && nblocks > kMaxBlocks) e = cudaErrorInvalidConfiguration;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + kOffBoxIn, boxes, sizeof(qk_box) * nbox, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    noalloc_table_kernel<<<1, 1, 0, s>>>(base, nbox, nghost);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    Geometry g{};
    g.boxes = reinterpret_cast<const DevBox *>(base + kOffDevBox);
    g.tiles = nullptr;
    g.ntiles = 0;
    g.nbox = nbox;
    g.ng = nghost;
    g.ncells = ncells;
    g.box_cell0 = reinterpret_cast<const long long *>(base + kOffPrefix);
    e = launch_sums(precision == QK_FP32_MIXED, g, *p, hydro, rad,
                    reinterpret_cast<double *>(base + kOffPartials), nblocks,
                    reinterpret_cast<double *>(base + kOffOut), s);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, base + kOffOut, sizeof(double) * QK_NSUMS, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    if (err && errlen > 0)
      snprintf(err, (size_t)errlen, "qk_conserved_sums_noalloc: %s", cudaGetErrorString(e));
    return QK_ECUDA;
  }
  return QK_OK;
}
