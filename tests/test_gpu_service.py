"""GPU tests of the continuous-batching service: results equal the stand-alone
builds alone and in the mix (tolerance: 1e-12 relative to max, the order of
atomic additions differs), admission by HBM budget, cancellation, bounded
waits and an injected admission failure that leaves the others intact."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_05622_gb300 import workloads as W  # noqa: E402

TOL = 1e-12


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_05622_gb300 import ltjk
    ltjk.lib()
    return ltjk


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def molecules():
    out = []
    for nh, nH, seed in ((1, 1, 1), (2, 2, 2), (3, 1, 3)):
        c, k = W.chain(nh, nH)
        out.append(W.build_molecule(c, k, W.draw_kind_bases(np.random.default_rng(seed))))
    return out


def test_mix_equals_alone(L):
    mols = molecules()
    ctxs = [L.Context(m, schwarz_tau=1e-12, precision=(L.MIXED if i == 1 else L.FP64))
            for i, m in enumerate(mols)]
    rng = np.random.default_rng(0)
    reqs = []
    for i, (m, c) in enumerate(zip(mols, ctxs)):
        D = dev(rng.standard_normal((5 + 3 * i, m.nao, m.nao)))
        J0, K0 = c.jk_build(D)
        P = dev(rng.standard_normal((2, m.nao, m.nao)))
        Q = dev(rng.standard_normal((2, m.nao, m.nao)))
        g0 = c.jk_grad(P, Q, 1.0, -0.5)
        reqs.append((c, D, J0, K0, P, Q, g0))
    torch.cuda.synchronize()
    svc = L.Service(1 << 30)
    tickets = []
    for (c, D, J0, K0, P, Q, g0) in reqs * 2:  # every request twice, all in flight together
        tj, J, K = svc.submit_jk(c, D)
        tg, g = svc.submit_grad(c, P, Q, 1.0, -0.5)
        tickets.append((tj, J, K, J0, K0, tg, g, g0))
    for (tj, J, K, J0, K0, tg, g, g0) in tickets:
        svc.wait(tj, 120)
        svc.wait(tg, 120)
        assert rel(J, J0) < TOL and rel(K, K0) < TOL
        assert rel(g, g0) < TOL
    st = svc.stats()
    assert st["completed"] == 2 * len(tickets) and st["failed"] == 0
    assert st["bytes_in_use"] == 0 and st["p99_ms"] >= st["p50_ms"] > 0
    svc.close()


def test_budget_admission_and_faults(L):
    m = molecules()[1]
    c = L.Context(m, schwarz_tau=1e-12)
    N = m.nao
    D = dev(np.random.default_rng(1).standard_normal((4, N, N)))
    J0, K0 = c.jk_build(D)
    torch.cuda.synchronize()
    per_req = 4 * 4 * N * N * 8
    svc = L.Service(max(per_req + 4096, 1 << 20))  # room for one request at a time
    with pytest.raises(L.LtjkError) as e:
        svc.submit_jk(c, dev(np.zeros((400, N, N))))  # can never fit
    assert e.value.code == L.EBUDGET
    ts = [svc.submit_jk(c, D) for _ in range(4)]
    svc.cancel(ts[3][0])
    for t, J, K in ts[:3]:
        svc.wait(t, 120)
        assert rel(J, J0) < TOL and rel(K, K0) < TOL
    with pytest.raises(L.LtjkError) as e:
        svc.wait(ts[3][0], 120)
    assert e.value.code == L.ECANCELLED
    st = svc.stats()
    assert st["bytes_peak"] <= st["budget"] and st["bytes_in_use"] == 0
    # injected admission failure: that request fails, the next one is unaffected
    svc.fail_next_admission(1)
    t_bad, _, _ = svc.submit_jk(c, D)
    t_ok, J, K = svc.submit_jk(c, D)
    with pytest.raises(L.LtjkError) as e:
        svc.wait(t_bad, 60)
    assert e.value.code == L.ENOMEM
    svc.wait(t_ok, 120)
    assert rel(J, J0) < TOL
    # bounded wait on an unknown ticket and a zero timeout never block
    with pytest.raises(L.LtjkError):
        svc.wait(987654, 0.0)
    svc.close()
