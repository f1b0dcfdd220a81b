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


def test_request_admitted_while_another_runs(L):
    """Continuous batching, not a queue: a small request submitted while a
    large one's kernels are already on the device is admitted into the
    running steps and completes first; both equal their stand-alone builds."""
    w = W.config3()  # 445 AO: many more work items (so steps) than the scheduler runs ahead
    big = L.Context(w.mol, schwarz_tau=1e-12, precision=L.MIXED)
    Db = dev(np.random.default_rng(7).standard_normal((8, w.mol.nao, w.mol.nao)))
    Jb0, Kb0 = big.jk_build(Db)
    m = molecules()[0]
    small = L.Context(m, schwarz_tau=1e-12, precision=L.MIXED)
    Ds = dev(np.random.default_rng(8).standard_normal((4, m.nao, m.nao)))
    Js0, Ks0 = small.jk_build(Ds)
    torch.cuda.synchronize()
    svc = L.Service(1 << 32)
    tb, Jb, Kb = svc.submit_jk(big, Db)
    # wait until the large request is admitted and its first steps are launched
    import time
    t0 = time.time()
    while svc.stats()["steps"] < 1 and time.time() - t0 < 30:
        time.sleep(0.0005)
    done_b, _ = svc.poll(tb)
    st = svc.stats()
    assert not done_b and st["active"] >= 1
    ts, Js, Ks = svc.submit_jk(small, Ds)
    svc.wait(ts, 120)
    done_b_at_small, _ = svc.poll(tb)
    svc.wait(tb, 120)
    assert not done_b_at_small  # the small one did not wait for the large one
    assert rel(Js, Js0) < TOL and rel(Ks, Ks0) < TOL
    assert rel(Jb, Jb0) < TOL and rel(Kb, Kb0) < TOL
    svc.close()
