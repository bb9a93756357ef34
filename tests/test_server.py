"""Serving loop: admission, cancellation, bounded waits, and results in a mix.

Host-side failure handling needs no GPU: a server with no workers admits
requests but never runs them, so a wait on one must give up with
HPM_ERR_TIMEOUT, a queued request can be cancelled, and a request larger than
the whole device-memory budget is refused. On the GPU, every request solved in
a mix of concurrent requests must equal the same request solved alone, bit for
bit.
"""
import time

import numpy as np
import pytest

from paper_1906_10734_gb300 import inputs as I


@pytest.fixture(scope="module")
def hpm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_10734_gb300 import hpm as H
    return H


def host_request(n, seed=0):
    pos = I.uniform_cube(n, seed)
    return pos, I.equal_masses(n), np.zeros(n, np.float32), np.zeros((n, 3), np.float32)


def test_admission_cancel_and_bounded_wait_without_workers(hpm):
    sv = hpm.Server(workers=0, max_batch=4, hbm_budget_bytes=64 << 20)
    # a request whose estimated footprint exceeds the whole budget is refused
    with pytest.raises(hpm.HpmError) as e:
        sv.submit(*host_request(1 << 20))
    assert e.value.status == -3
    t1 = sv.submit(*host_request(1000, 1))
    t2 = sv.submit(*host_request(1000, 2))
    assert sv.poll(t1)[0] == 0
    # nothing runs the queue: the bounded wait gives up
    t0 = time.perf_counter()
    with pytest.raises(hpm.HpmError) as e:
        sv.wait(t1, timeout_ms=200)
    assert e.value.status == -5 and 0.15 < time.perf_counter() - t0 < 5.0
    sv.cancel(t2)
    assert sv.poll(t2)[0] == -1
    with pytest.raises(hpm.HpmError):
        sv.wait(t2, timeout_ms=10)
    st = sv.stats()
    assert st["submitted"] == 2 and st["rejected"] == 1 and st["cancelled"] == 1 and st["queued"] == 1
    sv.close()


def test_tickets_end_with_their_final_state_and_destroy_wakes_waiters(hpm):
    import threading
    sv = hpm.Server(workers=0, max_batch=4, hbm_budget_bytes=64 << 20)
    t1 = sv.submit(*host_request(500, 3))
    t2 = sv.submit(*host_request(500, 4))
    sv.cancel(t1)
    # the cancelled request left the queue at once; its final state is reported
    # once, after which the server has forgotten the ticket
    assert sv.stats()["queued"] == 1
    assert sv.poll(t1)[0] == -1
    with pytest.raises(hpm.HpmError) as e:
        sv.poll(t1)
    assert e.value.status == -1
    # a thread blocked on a request nothing will run is woken by destroy and
    # told the server is going away (HPM_ERR_BUSY) before anything is freed
    got = {}

    def waiter():
        try:
            sv.wait(t2, timeout_ms=60000)
            got["status"] = 0
        except hpm.HpmError as err:
            got["status"] = err.status

    th = threading.Thread(target=waiter)
    th.start()
    time.sleep(0.2)
    t0 = time.perf_counter()
    sv.close()
    th.join(timeout=10)
    assert not th.is_alive() and got["status"] == -7 and time.perf_counter() - t0 < 5.0


@pytest.mark.gpu
def test_results_in_a_mix_equal_each_request_alone(hpm):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    ws = [I.batch_problem(k, 2000, 60000, 5) for k in range(24)]
    sv = hpm.Server(workers=2, max_batch=6)
    outs, tickets = [], []
    for k, w in enumerate(ws):
        if k % 2:   # device buffers
            b = (torch.from_numpy(w.pos).to(dev), torch.from_numpy(w.mass).to(dev),
                 torch.zeros(w.n, dtype=torch.float32, device=dev),
                 torch.zeros((w.n, 3), dtype=torch.float32, device=dev))
        else:       # host buffers
            b = (np.ascontiguousarray(w.pos), np.ascontiguousarray(w.mass), np.zeros(w.n, np.float32),
                 np.zeros((w.n, 3), np.float32))
        outs.append(b)
        tickets.append(sv.submit(*b))
        if k % 5 == 4:
            time.sleep(0.01)   # arrivals while earlier batches run
    lat = [sv.wait(t, 120000) for t in tickets]
    st = sv.stats()
    sv.close()
    assert st["completed"] == len(ws) and st["batches"] >= 2 and st["p99_ms"] >= st["p50_ms"] > 0
    assert all(x > 0 for x in lat)
    for w, b in zip(ws, outs):
        s = hpm.Solver(w.max_depth, w.ng, w.eps, w.leaf_max)
        phi, acc = s(torch.from_numpy(w.pos).to(dev), torch.from_numpy(w.mass).to(dev))
        torch.cuda.synchronize()
        s.close()
        got_phi = b[2].cpu().numpy() if hasattr(b[2], "cpu") else b[2]
        got_acc = b[3].cpu().numpy() if hasattr(b[3], "cpu") else b[3]
        assert np.array_equal(got_phi, phi.cpu().numpy())
        assert np.array_equal(got_acc, acc.cpu().numpy())


@pytest.mark.gpu
def test_budget_bounds_concurrency_and_all_requests_finish(hpm):
    ws = [I.batch_problem(k, 20000, 40000, 6) for k in range(6)]
    # room for one request at a time at a fixed 512 bytes per particle: batches of
    # one, served one after another
    sv = hpm.Server(workers=2, max_batch=8, hbm_budget_bytes=40000 * 512 + (8 << 20) + 1, bytes_per_particle=512.0)
    bufs = [(np.ascontiguousarray(w.pos), np.ascontiguousarray(w.mass), np.zeros(w.n, np.float32),
             np.zeros((w.n, 3), np.float32)) for w in ws]
    ts = [sv.submit(*b) for b in bufs]
    for t in ts:
        sv.wait(t, 120000)
    st = sv.stats()
    sv.close()
    assert st["completed"] == 6 and st["batches"] == 6
    assert all(np.abs(b[3]).sum() > 0 for b in bufs)


@pytest.mark.gpu
def test_admission_is_calibrated_from_measured_batches(hpm):
    """With no fixed rate the server measures each completed batch's device need (its
    plan's work buffers and packed buffers over its particles) and takes the largest;
    a single-request batch needs what a plan solving that request alone reports."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    w = I.batch_problem(3, 50000, 50001, 7)
    sv = hpm.Server(workers=1, max_batch=1)
    b = (np.ascontiguousarray(w.pos), np.ascontiguousarray(w.mass), np.zeros(w.n, np.float32),
         np.zeros((w.n, 3), np.float32))
    assert sv.stats()["bytes_per_particle"] == 0.0
    sv.wait(sv.submit(*b), 120000)
    rate = sv.stats()["bytes_per_particle"]
    sv.close()
    s = hpm.Solver(w.max_depth, w.ng, w.eps, w.leaf_max)
    s(torch.from_numpy(w.pos).to(dev), torch.from_numpy(w.mass).to(dev))
    torch.cuda.synchronize()
    st = hpm.hpm_get_stats(s.plan)
    s.close()
    packed = w.n * (24 + 8 + 4 + 12)
    assert st["table_bytes"] > 0 and st["work_bytes"] > 0
    # the batched build adds its problem-offset buffers to the single solve's need
    need = (st["work_bytes"] + packed - (8 << 20)) / w.n
    assert need <= rate < need + 64.0


@pytest.mark.gpu
def test_particle_bound_splits_batches(hpm):
    """With a bound of particles per batch no two of these requests share a batch (each
    is over half the bound), and a request over the bound still runs (alone)."""
    ws = [I.batch_problem(k, 20000, 30000, 9) for k in range(5)]
    sv = hpm.Server(workers=1, max_batch=8, max_batch_particles=35000)
    bufs = [(np.ascontiguousarray(w.pos), np.ascontiguousarray(w.mass), np.zeros(w.n, np.float32),
             np.zeros((w.n, 3), np.float32)) for w in ws]
    big = host_request(40000, 10)
    ts = [sv.submit(*b) for b in bufs] + [sv.submit(*big)]
    for t in ts:
        sv.wait(t, 120000)
    st = sv.stats()
    sv.close()
    assert st["completed"] == 6 and st["batches"] == 6
    assert all(np.abs(b[3]).sum() > 0 for b in bufs + [big])


def test_admission_uses_a_fixed_rate(hpm):
    """A caller's fixed rate replaces the calibrated estimate at submit (host logic,
    no workers): 4096 bytes per particle puts 20,000 particles over a 64 MiB budget."""
    sv = hpm.Server(workers=0, max_batch=4, hbm_budget_bytes=64 << 20, bytes_per_particle=4096.0)
    with pytest.raises(hpm.HpmError) as e:
        sv.submit(*host_request(20000, 1))   # 4096 x 20000 + 8 MiB > 64 MiB
    assert e.value.status == -3
    t = sv.submit(*host_request(10000, 2))
    assert sv.poll(t)[0] == 0
    sv.close()


@pytest.mark.gpu
def test_a_request_over_the_budget_after_calibration_runs_alone(hpm):
    """Requests accepted under the 512-byte prior are not stranded when the first
    batch's measurement raises the estimate above the whole budget: each runs alone
    once nothing else is in flight."""
    ws = [I.batch_problem(k, 30000, 30001, 8) for k in range(3)]
    n = max(w.n for w in ws)
    sv = hpm.Server(workers=1, max_batch=4, hbm_budget_bytes=512 * n + (8 << 20) + 1)
    bufs = [(np.ascontiguousarray(w.pos), np.ascontiguousarray(w.mass), np.zeros(w.n, np.float32),
             np.zeros((w.n, 3), np.float32)) for w in ws]
    ts = [sv.submit(*b) for b in bufs]
    for t in ts:
        sv.wait(t, 120000)
    st = sv.stats()
    sv.close()
    assert st["completed"] == 3 and st["batches"] == 3 and st["bytes_per_particle"] > 0
    assert all(np.abs(b[3]).sum() > 0 for b in bufs)
