"""The FP64 reciprocal and square root of the stage kernels against IEEE
results (numpy's correctly rounded division and square root): every result
within one ulp, on the argument ranges the kernels see (the Levermore
closure's [1, 4], the HLL wavespeed's (0, 1], densities and pressures over
many decades) and across the exponent range."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _args():
    rng = np.random.Generator(np.random.Philox(97))
    parts = [
        rng.uniform(1.0, 4.0, 200_000),                    # 4 - 3 |f|^2
        rng.uniform(0.0, 1.0, 200_000) + 1e-300,           # T_DD
        10.0 ** rng.uniform(-300, 300, 400_000),           # any magnitude
        np.nextafter(np.array([1.0, 2.0, 4.0, 0.25]), 0.0),
        np.array([1.0, 2.0, 3.0, 4.0, 0.5, 1e-300, 1e300, 1.0 / 3.0]),
    ]
    return np.concatenate(parts)


def _ulp_err(got, ref):
    return np.abs(got - ref) / np.spacing(np.abs(ref))


def test_reciprocal_and_sqrt_within_one_ulp(torch_cuda):
    torch = torch_cuda
    from paper_2110_01792_gb300 import qk
    x = _args()
    dx = torch.from_numpy(x).cuda()
    r = torch.empty_like(dx)
    s = torch.empty_like(dx)
    qk.eval_math(dx, r, s)
    torch.cuda.synchronize()
    er = _ulp_err(r.cpu().numpy(), 1.0 / x)
    es = _ulp_err(s.cpu().numpy(), np.sqrt(x))
    assert er.max() <= 1.0, (er.max(), x[np.argmax(er)])
    assert es.max() <= 1.0, (es.max(), x[np.argmax(es)])
    # mostly correctly rounded (the square root carries the rounding of its
    # first product x y, up to half an ulp, on top of the final rounding)
    assert np.mean(er <= 0.5) > 0.99 and np.mean(es <= 0.5) > 0.8


def test_sqrt_of_zero_is_zero(torch_cuda):
    torch = torch_cuda
    from paper_2110_01792_gb300 import qk
    dx = torch.tensor([0.0, 4.0], dtype=torch.float64, device="cuda")
    s = torch.empty_like(dx)
    qk.eval_math(dx, None, s)
    assert s.cpu().tolist() == [0.0, 2.0]


def test_integer_pipe_conversions(torch_cuda):
    """float -> double widening equals numpy's exact conversion for every
    class of float (normal, subnormal, zero, infinite, NaN); double -> float
    truncation lies within one FP32 ulp toward zero, flushes magnitudes below
    the normal float range to signed zeros and clamps above it."""
    torch = torch_cuda
    from paper_2110_01792_gb300 import qk
    rng = np.random.Generator(np.random.Philox(11))
    bits = rng.integers(0, 2 ** 32, 400_000, dtype=np.uint64).astype(np.uint32)
    extra = np.array([0.0, -0.0, np.inf, -np.inf, 1e-45, -1e-45, 1.17e-38, 3.4e38],
                     dtype=np.float32)
    f = np.concatenate([bits.view(np.float32), extra])
    d = torch.empty(f.size, dtype=torch.float64, device="cuda")
    qk.eval_convert(f_in=torch.from_numpy(f).cuda(), d_out=d)
    got = d.cpu().numpy()
    with np.errstate(invalid="ignore"):  # signalling NaN bit patterns
        ref = f.astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint64), ref[~nan].view(np.uint64))
    x = np.concatenate([rng.standard_normal(200_000) * 10.0 ** rng.uniform(-45, 45, 200_000),
                        np.array([0.0, -0.0, 1e300, -1e300, 1e-300, np.inf])])
    fo = torch.empty(x.size, dtype=torch.float32, device="cuda")
    qk.eval_convert(d_in=torch.from_numpy(x).cuda(), f_out=fo)
    y = fo.cpu().numpy().astype(np.float64)
    fmax, fmin = float(np.finfo(np.float32).max), float(np.finfo(np.float32).tiny)
    ax = np.abs(x)
    normal = (ax >= fmin) & (ax <= fmax)
    assert np.all(np.abs(y[normal]) <= ax[normal])
    up = np.nextafter(np.abs(y[normal]).astype(np.float32), np.float32(np.inf)).astype(np.float64)
    assert np.all(ax[normal] < up)
    assert np.all(np.sign(y[normal]) == np.sign(x[normal]))
    assert np.all(y[ax < fmin] == 0.0)
    big = np.isfinite(x) & (ax > fmax)
    assert np.all(np.abs(y[big]) == fmax)
    assert np.isinf(y[-1])


@pytest.mark.parametrize("fp64", [True, False], ids=["fp64", "fp32"])
def test_fma_probe_values_and_flop_count(torch_cuda, fp64):
    """The ALU probe computes what it counts: every thread's 8 chains
    a <- a (1 - 2^-20) + 2^-10 from a0 = (thread mod 32) + chain follow the
    closed form a_n = L + m^n (a0 - L), L = 2^-10 / 2^-20 = 1024 (rounding
    accumulates to ~n ulp(1024) at most), and the flop count is
    2 x 8 x iters x threads."""
    torch = torch_cuda
    from paper_2110_01792_gb300 import qk
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    n_threads = 8 * 256 * nsm
    sink = torch.full((n_threads + 100,), -1.0, dtype=torch.float64 if fp64 else torch.float32,
                      device="cuda")
    iters = 1000
    fl = qk.fma_probe(fp64, iters, sink)
    torch.cuda.synchronize()
    assert fl == 2.0 * 8 * iters * n_threads
    got = sink.double().cpu().numpy()
    m, L = 1.0 - 2.0 ** -20, 1024.0
    t = np.arange(n_threads) % 32
    exp = sum(L + m ** iters * ((t + i) - L) for i in range(8))
    ulp = np.spacing(np.float64(L) if fp64 else np.float32(L))
    assert np.max(np.abs(got[:n_threads] - exp)) <= 8 * iters * float(ulp)
    assert np.all(got[n_threads:] == -1.0)  # nothing beyond the launched threads
    with pytest.raises(qk.QKError):
        qk.fma_probe(fp64, 0, sink)
