"""Request server: continuous batching, budget admission, cancellation,
bounded waits; each result is the same alone and in the mix."""
import numpy as np
import pytest

import parity as P
from paper_1110_4903_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1110_4903_gb300 import chem
    m9, m36 = synth.h2_air_9sp(), synth.hydrocarbon_36sp()
    h9 = chem.Chem(m9, precision=chem.MIXED)
    h36 = chem.Chem(m36, precision=chem.MIXED)
    yield torch, chem, {9: (m9, h9), 36: (m36, h36)}
    h9.close()
    h36.close()


def _wait(srv, t, timeout_s=60.0):
    """A bounded wait: a request the server never finishes fails the test."""
    res = srv.wait(t, timeout_us=int(timeout_s * 1e6))
    assert res is not None, "request %d did not finish within %.0f s" % (t, timeout_s)
    return res


def _states(torch, mech, n, seed):
    f = synth.uniform_field(mech.ns, n, 900.0, 2800.0, seed=seed)
    rho, e = P.initial_state(mech, f)
    dev = torch.device("cuda")
    return torch.tensor(rho, device=dev), torch.tensor(e, device=dev)


def _requests(torch, mechs):
    rng = np.random.default_rng(5)
    out = []
    for i in range(16):
        ns = 9 if i % 2 == 0 else 36
        n = int(np.exp(rng.uniform(np.log(300), np.log(20000 if ns == 9 else 3000))))
        dt = float(np.exp(rng.uniform(np.log(1e-8), np.log(1e-5))))
        rho, e = _states(torch, mechs[ns][0], n, seed=1000 + i)
        out.append((ns, rho, e, dt))
    return out


def test_alone_equals_mixed(env):
    torch, chem, mechs = env
    reqs = _requests(torch, mechs)
    # alone: one request at a time through the server
    srv = chem.Server(max_inflight=8)
    alone = []
    for ns, rho, e, dt in reqs:
        r, ev = rho.clone(), e.clone()
        t = srv.submit(mechs[ns][1], r, ev, dt)
        res = _wait(srv, t)
        assert res.state == chem.REQ_DONE
        alone.append((r, ev))
    # mixed: all submitted at once, overlapping on the device
    mixed = []
    tickets = []
    for ns, rho, e, dt in reqs:
        r, ev = rho.clone(), e.clone()
        tickets.append(srv.submit(mechs[ns][1], r, ev, dt))
        mixed.append((r, ev))
    spans = []
    for t in tickets:
        res = _wait(srv, t)
        assert res.state == chem.REQ_DONE
        assert 0 < res.dev_first_ns <= res.dev_last_ns
        spans.append((res.dev_first_ns, res.dev_last_ns))
    # several requests had cells on the device at the same time (device clock)
    overlap = sum(1 for i in range(len(spans)) for j in range(i)
                  if spans[i][0] < spans[j][1] and spans[j][0] < spans[i][1])
    assert overlap > 0
    for (ra, ea), (rm, em) in zip(alone, mixed):
        assert torch.equal(ra, rm) and torch.equal(ea, em)
    # and the server's result is chem_advance's
    ns, rho, e, dt = reqs[1]
    r, ev = rho.clone(), e.clone()
    mechs[ns][1].advance(r, ev, dt)
    torch.cuda.synchronize()
    assert torch.equal(r, mixed[1][0])
    st = srv.stats()
    assert st["failed"] == 0 and st["completed"] == 2 * len(reqs) and st["bytes_in_use"] == 0
    srv.close()


def test_ring_laps_and_chunk_edges(env):
    """More chunks than the descriptor ring holds, so its entries and their
    claim counters go round more than one lap, with request sizes at the
    chunk edges (1, 1023, 1024, 1025 cells, ...): every result equals a
    direct step of the same cells, and the queue reports no error."""
    torch, chem, mechs = env
    m, h = mechs[9]
    sizes = [1, 2, 1023, 1024, 1025, 2047, 2048, 2049, 3000]   # 16 chunks a round
    rho0, e0 = _states(torch, m, max(sizes), seed=77)
    dt = 1e-7
    refs = {}
    for n in sizes:
        r, e = rho0[:, :n].clone(), e0[:n].clone()
        h.advance(r, e, dt)
        refs[n] = (r, e)
    torch.cuda.synchronize()
    srv = chem.Server(max_inflight=64)
    rounds = 72   # 1,152 chunks: past the 1,024 ring entries
    for k in range(rounds):
        outs, tickets = [], []
        for n in sizes:
            r, e = rho0[:, :n].clone(), e0[:n].clone()
            tickets.append(srv.submit(h, r, e, dt))
            outs.append((n, r, e))
        for t in tickets:
            res = srv.wait(t, timeout_us=20_000_000)
            assert res is not None and res.state == chem.REQ_DONE
        for n, r, e in outs:
            assert torch.equal(r, refs[n][0]) and torch.equal(e, refs[n][1]), (k, n)
    st = srv.stats()
    assert st["failed"] == 0 and st["completed"] == rounds * len(sizes)
    assert st["queue_errors"] == 0
    srv.close()


def test_many_one_cell_requests(env):
    """A stream of requests of one cell each: every chunk holds a single
    real cell, so the host's publication window has to follow the kernels'
    hand-out of chunks, not of cells (a window that waited for claims to
    cross cell boundaries stalled here).  Bounded waits: a stall fails the
    test instead of hanging it."""
    torch, chem, mechs = env
    m, h = mechs[9]
    rho0, e0 = _states(torch, m, 1, seed=78)
    dt = 1e-7
    r_ref, e_ref = rho0.clone(), e0.clone()
    h.advance(r_ref, e_ref, dt)
    torch.cuda.synchronize()
    srv = chem.Server(max_inflight=64)
    outs = []
    for _ in range(300):
        r, e = rho0.clone(), e0.clone()
        outs.append((srv.submit(h, r, e, dt), r, e))
    for t, r, e in outs:
        res = srv.wait(t, timeout_us=20_000_000)
        assert res is not None and res.state == chem.REQ_DONE
        assert torch.equal(r, r_ref) and torch.equal(e, e_ref)
    st = srv.stats()
    assert st["failed"] == 0 and st["queue_errors"] == 0
    srv.close()


def test_small_requests_join_a_running_grid(env):
    """Continuous batching on the device: small requests submitted while a
    large one of the same mechanism runs are claimed by slots that free up
    inside the running grid -- their first cell starts and their last cell
    finishes before the large request's last cell (device clock) -- and each
    result equals chem_advance_ex's on the same input."""
    torch, chem, mechs = env
    m, h = mechs[36]
    big = _states(torch, m, 1 << 17, seed=11)
    smalls = [_states(torch, m, n, seed=200 + i) for i, n in enumerate([512, 800, 1000, 1500, 700, 2000, 900, 1200])]
    refs = []
    for r, e in smalls:
        rr, ee = r.clone(), e.clone()
        h.advance(rr, ee, 1e-6)
        refs.append((rr, ee))
    torch.cuda.synchronize()
    srv = chem.Server()
    launches0 = srv.stats()["launches"]
    rb, eb = big[0].clone(), big[1].clone()
    tb = srv.submit(h, rb, eb, 1e-6)
    import time
    time.sleep(0.03)                       # the large request is running
    assert srv.poll(tb).state == chem.REQ_RUNNING
    work = [(r.clone(), e.clone()) for r, e in smalls]
    ts = [srv.submit(h, r, e, 1e-6) for r, e in work]
    res_b = _wait(srv, tb)
    assert res_b.state == chem.REQ_DONE
    inside = 0
    for t, (r, e), (rr, ee) in zip(ts, work, refs):
        res = _wait(srv, t)
        assert res.state == chem.REQ_DONE
        assert torch.equal(r, rr) and torch.equal(e, ee)
        assert res.dev_first_ns > res_b.dev_first_ns
        inside += res.dev_last_ns < res_b.dev_last_ns
    assert inside == len(ts), inside
    st = srv.stats()
    # one lane, one kernel instance carried the large and the small requests
    assert st["launches"] - launches0 == 1 and st["queue_errors"] == 0
    srv.close()


def test_two_mechanisms_share_the_device(env):
    """Small requests of a second mechanism get a share of the GPU while a
    large request of the first runs: they finish before it does."""
    torch, chem, mechs = env
    m36, h36 = mechs[36]
    m9, h9 = mechs[9]
    big = _states(torch, m36, 1 << 17, seed=12)
    smalls = [_states(torch, m9, n, seed=300 + i) for i, n in enumerate([4000, 9000, 6000, 12000])]
    # (references first: a plain launch cannot start while the server's
    # persistent kernel holds the SMs)
    refs = []
    for r, e in smalls:
        rr, ee = r.clone(), e.clone()
        h9.advance(rr, ee, 1e-6)
        refs.append((rr, ee))
    torch.cuda.synchronize()
    srv = chem.Server()
    tb = srv.submit(h36, big[0], big[1], 1e-6)
    import time
    time.sleep(0.03)
    assert srv.poll(tb).state == chem.REQ_RUNNING
    ts = [srv.submit(h9, r, e, 1e-6) for r, e in smalls]
    res_b = _wait(srv, tb)
    for t, (r, e), (rr, ee) in zip(ts, smalls, refs):
        res = _wait(srv, t)
        assert res.state == chem.REQ_DONE
        assert res.dev_last_ns < res_b.dev_last_ns
        assert torch.equal(r, rr) and torch.equal(e, ee)
    assert srv.stats()["queue_errors"] == 0
    srv.close()


def test_host_requests_match_device(env):
    torch, chem, mechs = env
    m, h = mechs[9]
    rho, e = _states(torch, m, 5000, seed=7)
    srv = chem.Server()
    r_dev, e_dev = rho.clone(), e.clone()
    _wait(srv, srv.submit(h, r_dev, e_dev, 1e-6))
    r_h, e_h = rho.cpu().numpy().copy(), e.cpu().numpy().copy()
    status = np.full(5000, -1, np.int32)
    res = _wait(srv, srv.submit(h, r_h, e_h, 1e-6, host=True, status=status))
    assert res.state == chem.REQ_DONE
    assert np.array_equal(r_h, r_dev.cpu().numpy()) and np.array_equal(e_h, e_dev.cpu().numpy())
    assert (status == 0).all()
    srv.close()


def test_budget_admission_and_refusal(env):
    torch, chem, mechs = env
    m, h = mechs[36]
    per_cell = 8 * m.ns + 20
    sizes = [2000, 1500, 2500, 1000, 3000, 2200]
    budget = int(max(sizes) * per_cell + 1024) * 2          # about two requests at a time
    srv = chem.Server(budget_bytes=budget, max_inflight=8)
    states = [_states(torch, m, n, seed=50 + i) for i, n in enumerate(sizes)]
    tickets = [srv.submit(h, r, e, 1e-6) for r, e in states]
    peak = 0
    while True:
        st = srv.stats()
        assert st["bytes_in_use"] <= st["budget_bytes"]
        peak = max(peak, st["running"])
        if st["completed"] == len(sizes):
            break
    assert peak <= 3
    for t in tickets:
        assert srv.poll(t).state == chem.REQ_DONE
    big = _states(torch, m, int(budget / per_cell) + 100, seed=99)
    with pytest.raises(chem.ChemError) as ei:
        srv.submit(h, big[0], big[1], 1e-6)
    assert ei.value.code == -4
    srv.close()


def test_cancel_wait_timeout_and_errors(env):
    torch, chem, mechs = env
    m, h = mechs[36]
    srv = chem.Server(max_inflight=1)
    long_r, long_e = _states(torch, m, 20000, seed=3)
    t_long = srv.submit(h, long_r, long_e, 1e-6)
    q_r, q_e = _states(torch, m, 500, seed=4)
    q_r0, q_e0 = q_r.clone(), q_e.clone()
    t_q = srv.submit(h, q_r, q_e, 1e-6)
    c_state = _states(torch, m, 500, seed=5)
    c0 = c_state[0].clone()
    t_c = srv.submit(h, c_state[0], c_state[1], 1e-6)
    assert srv.wait(t_q, timeout_us=1) is None                 # still queued behind t_long
    srv.cancel(t_c)
    assert srv.poll(t_c).state == chem.REQ_CANCELLED
    assert _wait(srv, t_q).state == chem.REQ_DONE
    assert _wait(srv, t_long).state == chem.REQ_DONE
    assert not torch.equal(q_r, q_r0)
    assert torch.equal(c_state[0], c0)                         # the cancelled state is untouched
    with pytest.raises(chem.ChemError) as ei:
        srv.cancel(t_q)                                        # finished: not cancellable
    assert ei.value.code == -1
    with pytest.raises(chem.ChemError) as ei:
        srv.poll(123456789)
    assert ei.value.code == -8
    with pytest.raises(chem.ChemError) as ei:
        srv.submit(h, q_r, q_e, -1.0)
    assert ei.value.code == -1
    srv.release(t_q)
    with pytest.raises(chem.ChemError):
        srv.poll(t_q)
    # destroying a server with queued work cancels it and returns
    keep = [_states(torch, m, 4000, seed=60 + i) for i in range(4)]
    for r, e in keep:
        srv.submit(h, r, e, 1e-6)
    srv.close()
    torch.cuda.synchronize()
