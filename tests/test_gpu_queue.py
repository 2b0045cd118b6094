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


def _batch_alone(case, k):
    import paper_2110_10765_gb300 as ci
    a = _args(case)
    b = ci.Batch([ci.Problem(a["sp"], a["Z"], a["N"], a["nmax"], a["twoM"], a["eps"], seed=a["seed"])], k=[k])
    b.run()
    return b.result(0)[0]


# a large request (3 protons, 5 neutrons in shells N <= 3, Nmax 4: dim
# 116,184) that keeps running while the others are submitted
BIG = (3, 3, 5, 4, 21)


def test_queue_matches_batch_and_overlaps():
    """Requests submitted while a large one runs are admitted before it
    finishes (their engine steps are shared with it), and every result is
    bit-identical to the same problem solved alone in a batch."""
    import paper_2110_10765_gb300 as ci
    ks = [5, 3, 6, 4, 2, 5, 4]
    ref_big = _batch_alone(BIG, 5)
    ref = [_batch_alone(c, k) for c, k in zip(CASES, ks)]
    q = ci.Queue(max_slots=4)
    big = q.submit(k=5, **_args(BIG))
    t0 = time.time()
    while q.stats()["admitted"] < 1:       # the large request is on the GPU
        assert time.time() - t0 < 60
        time.sleep(0.001)
    st, rb = q.poll(big)
    assert st == 6, "the large request finished before the others were submitted"
    steps_before = q.stats()["steps"]
    late = [q.submit(k=ks[i], **_args(CASES[i])) for i in range(len(CASES))]
    res = _wait(q, [big] + late)
    st, rb = res[big]
    assert st == 0, rb
    assert np.array_equal(rb["evals"], ref_big), rb["evals"] - ref_big
    for i, t in enumerate(late):
        st, r = res[t]
        assert st == 0, r
        assert np.array_equal(r["evals"], ref[i]), (i, r["evals"] - ref[i])
        assert r["t_done"] >= r["t_admit"] >= r["t_submit"] and r["latency_s"] > 0
        assert max(r["residual"]) < 1e-3
        # admitted while the large request was still running: overlap
        assert r["t_admit"] < rb["t_done"], (i, r["t_admit"], rb["t_done"])
    s = q.stats()
    assert s["completed"] == len(CASES) + 1 and s["admitted"] == len(CASES) + 1
    assert s["steps"] > steps_before
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
    bad = q.submit(k=3, **_args((1, 1, 1, -1, 3)) | {"nmax": -1, "twoM": 9})   # empty basis
    st, r = _wait(q, [bad])[bad]
    assert st == 1   # CI_ERR_INVALID_ARG
    q.close()


@pytest.mark.parametrize("case,k", [((1, 1, 1, -1, 3), 2), ((1, 2, 1, -1, 4), 5), ((2, 1, 1, 0, 5), 1)])
def test_queue_solves_small_requests(case, k):
    """Spaces too small for the engine's Krylov blocks (dimension <= 80) are
    solved on the single-problem path inside the queue, beside a running
    engine request, and match the oracle's dense eigenvalues."""
    import oracle
    import paper_2110_10765_gb300 as ci
    from helpers import EIG_REL, oracle_problem
    a = _args(case)
    q = ci.Queue(max_slots=2)
    running = q.submit(k=3, **_args(CASES[1]))
    t = q.submit(k=k, **a)
    res = _wait(q, [running, t])
    st, r = res[t]
    assert st == 0, r
    assert 0 < r["dim"] <= 80
    T = synth.tbme_tables(a["sp"], a["seed"], np.float32)
    inp = dict(sp=a["sp"], Z=a["Z"], N=a["N"], nmax=a["nmax"], twoM=a["twoM"], eps=a["eps"], tables=T)
    o = oracle_problem(inp)
    ref = oracle.lowest_dense(oracle.dense_from_csr(*o.csr()[:3], o.dim), k)
    assert np.all(np.abs(r["evals"] - ref) <= EIG_REL * np.maximum(np.abs(ref), 1)), r["evals"] - ref
    assert res[running][0] == 0
    q.close()
