"""Serving queue with continuous batching: results equal the batched solve
of the same problem (alone or mixed), requests submitted while others run
complete, the memory budget refuses what cannot fit, cancellation."""

import time

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(2, 2, 3, 2, 11), (2, 3, 3, 2, 12), (3, 2, 2, 3, 13), (2, 2, 2, 4, 14), (3, 3, 2, 2, 15),
         (2, 4, 2, 2, 16), (2, 3, 2, 3, 17)]


def _args(case):
    n_shell, Z, N, nmax, seed = case
    sp = synth.ho_sp_table(n_shell)
    return dict(sp=sp, Z=Z, N=N, nmax=nmax, twoM=(Z + N) % 2, eps=synth.sp_energies(sp, 20.0), seed=seed)


def _wait(q, tickets, timeout=120.0):
    t0 = time.time()
    out = {}
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            st, r = q.poll(t)
            if st != 6:
                out[t] = (st, r)
        if time.time() - t0 > timeout:
            raise TimeoutError("queue did not finish")
        time.sleep(0.002)
    return out


def test_queue_matches_batch_and_overlaps():
    import paper_2110_10765_gb300 as ci
    ks = [5, 3, 6, 4, 2, 5, 4]
    # reference: each problem alone in a batch
    ref = []
    for c, k in zip(CASES, ks):
        a = _args(c)
        b = ci.Batch([ci.Problem(a["sp"], a["Z"], a["N"], a["nmax"], a["twoM"], a["eps"], seed=a["seed"])], k=[k])
        b.run()
        ref.append(b.result(0)[0])
    q = ci.Queue(max_slots=4)
    first = [q.submit(k=ks[i], **_args(CASES[i])) for i in range(3)]
    time.sleep(0.01)   # the rest arrives while the first ones run
    rest = [q.submit(k=ks[i], **_args(CASES[i])) for i in range(3, len(CASES))]
    res = _wait(q, first + rest)
    for i, t in enumerate(first + rest):
        st, r = res[t]
        assert st == 0, r
        assert np.array_equal(r["evals"], ref[i]), (i, r["evals"] - ref[i])
        assert r["t_done"] >= r["t_admit"] >= r["t_submit"] and r["latency_s"] > 0
        assert max(r["residual"]) < 1e-3
    s = q.stats()
    assert s["completed"] == len(CASES) and s["admitted"] == len(CASES)
    q.close()


def test_queue_refuses_requests_beyond_budget():
    import paper_2110_10765_gb300 as ci
    q = ci.Queue(mem_budget=1 << 20, max_slots=2)
    t = q.submit(k=3, **_args(CASES[1]))
    st, r = _wait(q, [t])[t]
    assert st == 4 and r["status"] == 4   # CI_ERR_CAPACITY
    q.close()


def test_queue_cancel_waiting_request():
    import paper_2110_10765_gb300 as ci
    q = ci.Queue(max_slots=1)
    running = q.submit(k=5, **_args(CASES[6]))
    waiting = q.submit(k=5, **_args(CASES[5]))
    q.cancel(waiting)
    res = _wait(q, [running, waiting])
    assert res[running][0] == 0
    assert res[waiting][0] in (0, 7)   # finished first, or CI_ERR_CANCELLED
    q.close()


def test_queue_rejects_bad_requests():
    import paper_2110_10765_gb300 as ci
    q = ci.Queue(max_slots=2)
    with pytest.raises(ci.CIError):
        q.submit(k=40, **_args(CASES[0]))
    small = _args((1, 1, 1, -1, 3))  # dimension 20: too small for the engine
    t = q.submit(k=2, **small)
    st, r = _wait(q, [t])[t]
    assert st == 1   # CI_ERR_INVALID_ARG
    q.close()
