"""The allocation-free J/K entry point, for callers that cannot let a library
allocate device memory (their own pool owns it, or cudaMalloc's implicit
synchronisation is unaffordable): two calls in a row through the C ABI must
reproduce ltjk_jk_build within the tests' FP64 tolerance, with the shared
fixed scratch array reused between the calls.  Collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_05622_gb300 import workloads as W  # noqa: E402

TOL64 = 1e-10


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_05622_gb300 import ltjk
    ltjk.lib()
    return ltjk


def rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_jk_build_twice(L, precision):
    wl = W.small_chain(2, 2, seed=4, tau=1e-12)
    prec = L.FP64 if precision == "fp64" else L.MIXED
    ctx = L.Context(wl.mol, schwarz_tau=1e-12, mixed_tau=1e-6, precision=prec)
    N = wl.mol.nao
    rng = np.random.default_rng(11)
    for call in range(2):  # second call reuses the array left by the first
        nd = 37 if call == 0 else 9
        D = torch.from_numpy(rng.standard_normal((nd, N, N))).to("cuda:0")
        J0, K0 = ctx.jk_build(D)
        J = torch.full_like(D, np.nan)
        K = torch.full_like(D, np.nan)
        ctx.jk_build_noalloc(D, J, K)
        torch.cuda.synchronize()
        assert rel(J, J0) <= TOL64 and rel(K, K0) <= TOL64, (call, rel(J, J0), rel(K, K0))


def test_noalloc_allocates_nothing(L):
    """In a fresh context, before any other build: the context's device memory
    does not grow, and after one warm-up call (which loads the kernels) a
    second call leaves the device's free memory unchanged."""
    wl = W.small_chain(2, 2, seed=4, tau=1e-12)
    ctx = L.Context(wl.mol, schwarz_tau=1e-12, mixed_tau=1e-6, precision=L.MIXED)
    N = wl.mol.nao
    D = torch.from_numpy(np.random.default_rng(13).standard_normal((8, N, N))).to("cuda:0")
    J, K = torch.empty_like(D), torch.empty_like(D)
    bytes0 = ctx.stats()["device_bytes"]
    ctx.jk_build_noalloc(D, J, K)
    torch.cuda.synchronize()
    assert ctx.stats()["device_bytes"] == bytes0
    free0 = torch.cuda.mem_get_info()[0]
    J2, K2 = torch.full_like(D, np.nan), torch.full_like(D, np.nan)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    ctx.jk_build_noalloc(D, J2, K2)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free1
    assert ctx.stats()["device_bytes"] == bytes0
    assert free0 >= free1
    J0, K0 = ctx.jk_build(D)  # the allocating build, afterwards
    torch.cuda.synchronize()
    assert rel(J2, J0) <= TOL64 and rel(K2, K0) <= TOL64
    assert rel(J, J0) <= TOL64 and rel(K, K0) <= TOL64


def test_noalloc_rejects_oversize(L):
    w = W.config2()
    ctx = L.Context(w.mol, schwarz_tau=1e-12)
    N = w.mol.nao
    D = torch.zeros((60, N, N), dtype=torch.float64, device="cuda:0")  # 4*60*200^2 > 8*2^20
    J, K = torch.empty_like(D), torch.empty_like(D)
    with pytest.raises(L.LtjkError) as e:
        ctx.jk_build_noalloc(D, J, K)
    assert e.value.code == L.EINVAL and "limit" in str(e.value)
