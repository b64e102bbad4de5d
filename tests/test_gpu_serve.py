"""Serving (continuous batching): results match the oracle, are bitwise the same alone and
in a mix, admission respects slots and the HBM budget, and errors come back as statuses."""

import time

import numpy as np
import pytest

import pfem_inputs as pi
from oracle import fem, solve
from tests.gpu_util import pfem, rel_l2

pytestmark = pytest.mark.gpu


def _requests():
    reqs = []
    for k, n in enumerate((5, 7, 9, 6)):
        p = pi.cube_problem(n, seed=100 + k)
        m = fem.Mesh(p)
        u_star, _, _ = solve.solve_linear(m, tol=1e-13)
        warm = pi.make_warm_start(p, u_star, seed=7 + k) if k % 2 else None
        reqs.append(dict(problem=p, u0=warm, solve="linear", steps=1, u_star=u_star))
    for k, dims in enumerate(((8, 2, 2), (12, 3, 3))):
        p = pi.bar_problem(*dims, seed=200 + k, stretch=0.1)
        m = fem.Mesh(p)
        u_star, _, _ = solve.solve_newton(m, tol=1e-12, n_load_steps=2, direct=True)
        warm = pi.make_warm_start(p, u_star, seed=9 + k) if k == 0 else None
        reqs.append(dict(problem=p, u0=warm, solve="newton", steps=1 if warm is not None else 2, u_star=u_star))
    return reqs


@pytest.fixture(scope="module")
def reqs():
    return _requests()


def _run(server, items, timeout=300.0):
    tickets = [server.submit(r["problem"], r["u0"], 1e-8, r["solve"], r["steps"]) for r in items]
    out = [None] * len(tickets)
    t0 = time.time()
    while any(o is None for o in out):
        for i, t in enumerate(tickets):
            if out[i] is None:
                out[i] = server.poll(t)
        if time.time() - t0 > timeout:
            raise TimeoutError("serving test did not finish")
        time.sleep(0.002)
    return out


def test_mix_matches_oracle_and_alone_bitwise(reqs):
    P = pfem()
    server = P.Server(8 << 30, max_slots=3)  # fewer slots than requests: continuous admission
    mixed = _run(server, reqs)
    server.close()
    for r, (st, u, info) in zip(reqs, mixed):
        assert st == 0, info
        assert rel_l2(u, r["u_star"]) <= 1e-6
        m = fem.Mesh(r["problem"])
        if r["solve"] == "linear":
            u_ref, it_ref, rel = solve.solve_linear(m, u0=r["u0"], tol=1e-8)
            assert abs(info["iterations"] - it_ref) <= max(2, int(0.015 * it_ref)), (info, it_ref)
            assert info["rel_residual_true_f64"] < 1e-8
        else:
            ref = solve.newton_reference(m, 1.0)
            assert np.linalg.norm(fem.residual(m, u)) <= 1.01e-8 * ref
        assert info["total_s"] >= info["queue_s"] >= 0.0
    for r, (st, u, info) in zip(reqs, mixed):
        alone_server = P.Server(8 << 30, max_slots=1)
        st2, u2, info2 = _run(alone_server, [r])[0]
        alone_server.close()
        assert st2 == 0 and np.array_equal(u, u2), "result differs alone vs in the mix"
        assert info["iterations"] == info2["iterations"]


def test_budget_admission_and_over_budget(reqs):
    P = pfem()
    big = reqs[2]["problem"]
    server = P.Server(64 << 10, max_slots=8)  # 64 KiB: the 9^3 cube can never fit
    t = server.submit(big, None, 1e-8)
    res = None
    for _ in range(5000):
        res = server.poll(t)
        if res is not None:
            break
        time.sleep(0.002)
    assert res is not None and res[0] == 7  # PFEM_ERR_OVER_BUDGET
    server.close()
    # one slot: requests run strictly one after another and all complete
    small = [reqs[0], reqs[3]]
    server = P.Server(1 << 30, max_slots=1)
    out = _run(server, small)
    server.close()
    assert all(o[0] == 0 for o in out)


def test_unknown_ticket_and_drain():
    P = pfem()
    from paper_2601_03086_gb300._lib import PfemError

    server = P.Server(1 << 30, max_slots=2)
    with pytest.raises(KeyError):
        server.poll(12345)
    p = pi.cube_problem(4, seed=1)
    t = server.submit(p)
    server.drain(120.0)
    st, u, info = server.poll(t)
    assert st == 0
    server.close()
    del PfemError


def test_bench_size_requests_match_oracle_alone_and_mixed():
    """Requests of the sizes the benchmark serves (~50k tets): a 20^3 cube (48,000 tets) zero
    and warm started, and a 48x12x12 Neo-Hookean bar (41,472 tets, 10% stretch) warm started.
    Served together they match the oracle (solutions within 1e-6, linear iteration counts
    within the FP32 bar) and are bitwise the results each gives alone."""
    P = pfem()
    items = []
    p = pi.cube_problem(20, seed=105)
    m = fem.Mesh(p)
    u_star, _, _ = solve.solve_linear(m, tol=1e-13)
    for warm in (None, pi.make_warm_start(p, u_star, seed=11)):
        items.append(dict(problem=p, u0=warm, solve="linear", steps=1, u_star=u_star))
    pb = pi.bar_problem(48, 12, 12, seed=205, stretch=0.1)
    mb = fem.Mesh(pb)
    u5, _, _ = solve.solve_newton(mb, tol=1e-8, n_load_steps=5)
    ub_star, _, _ = solve.solve_newton(mb, u0=u5, tol=1e-12, n_load_steps=1, inner_tol=1e-12)
    items.append(dict(problem=pb, u0=pi.make_warm_start(pb, ub_star, seed=13), solve="newton", steps=1,
                      u_star=ub_star))
    server = P.Server(16 << 30, max_slots=8)
    mixed = _run(server, items, timeout=600.0)
    server.close()
    for r, (st, u, info) in zip(items, mixed):
        assert st == 0, info
        assert rel_l2(u, r["u_star"]) <= 1e-6
        mm = fem.Mesh(r["problem"])
        if r["solve"] == "linear":
            _, it_ref, _ = solve.solve_linear(mm, u0=r["u0"], tol=1e-8)
            assert abs(info["iterations"] - it_ref) <= max(2, int(0.015 * it_ref)), (info, it_ref)
            assert info["rel_residual_true_f64"] < 1e-8
        else:
            _, n_ref, _ = solve.solve_newton(mm, u0=r["u0"], tol=1e-8, n_load_steps=1)
            assert abs(info["newton_iterations"] - n_ref) <= 2, (info, n_ref)
            assert np.linalg.norm(fem.residual(mm, u)) <= 1.01e-8 * solve.newton_reference(mm, 1.0)
    for r, (st, u, info) in zip(items, mixed):
        alone = P.Server(16 << 30, max_slots=1)
        st2, u2, info2 = _run(alone, [r], timeout=600.0)[0]
        alone.close()
        assert st2 == 0 and np.array_equal(u, u2), "result differs alone vs in the mix"
        assert info["iterations"] == info2["iterations"]
