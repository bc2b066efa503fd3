"""Tensor-core DST-I (split-BF16 digit products, tcgen05) vs the CPU oracle, through the C ABI (marked gpu).

The mixed path transforms Dirichlet grids whose sizes are multiples of 128 (up
to 1024, n + 1 not a power of two) with exact float32 sums of bf16 digit
products; its error is about 2^(-7k) for k digits (k from the plan's
tolerance), so results are held to 1e-9 relative here (the float64 path's bar
is 1e-11; the transform with tol 1e-10 keeps 6 digits, about 2^-42 per digit
product, summed over up to 1024 terms and two passes).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2603_04350_gb300 import inputs as I

from .test_gpu_parity import DEV, P, dev, host, relmax

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def expd():
    import __graft_entry__ as g
    g.build()
    from paper_2603_04350_gb300 import expd as E
    return E


# rectangular (slow axis 256, fast axis 128: a swapped axis would show), both
# multiples of 128, several 128-row tiles per slice and a slice count that
# leaves a ragged last wave of tiles
TC_CASES = [
    P("tc_d2d_s1", "dirichlet", (256, 128), 1, Nt=9),
    P("tc_d2d_s2", "dirichlet", (128, 256), 2, Nt=10),
    P("tc_d2d_s6", "dirichlet", (128, 128), 6, Nt=13),
    P("tc_d2d_ac_s1", "dirichlet", (128, 256), 1, nonlin="allen_cahn", a=0.01, c=0.0, dt=1e-3, Nt=12, alpha=1e-3),
    # 384 and 640 points: folded, S's halves have 192 or 320 rows, ending in
    # a half-filled 128-row tile (64-column products over three or five
    # 64-K steps)
    P("tc_d2d_640_s1", "dirichlet", (640, 128), 1, Nt=5),
    P("tc_d2d_384_s2", "dirichlet", (384, 256), 2, Nt=7),
]
TC_IDS = [p.name for p in TC_CASES]


def _counts(plan):
    return plan.timing_read(reset=True)["classes"]


TILES = [0, 8]          # 128 x 128 output tiles, 128 x 64 tiles (EXPD_KF_DST_N64)


@pytest.mark.parametrize("fold", ["1", "0"], ids=["folded", "full"])
@pytest.mark.parametrize("flags", TILES, ids=["n128", "n64"])
@pytest.mark.parametrize("p", TC_CASES, ids=TC_IDS)
def test_tc_residual_matches_oracle(expd, p, flags, fold, monkeypatch):
    # the residual of a mixed plan is float64 arithmetic around the two
    # transforms, so its error is the transforms' error; folded: the products
    # over the symmetric half of S (EXPD_DST_FOLD=1, the default), full: over
    # all of S
    monkeypatch.setenv("EXPD_DST_FOLD", fold)
    sp = O.spec_of(p)
    rng = np.random.default_rng(13)
    amp = 0.5 if p.nonlin != "none" else 1.0
    u0 = amp * rng.uniform(-1, 1, p.n)
    U = amp * rng.uniform(-1, 1, (p.Nt,) + p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    U_start = np.concatenate([u0[None], U[: p.order - 1]])
    ref = O.residual(sp, U[p.order - 1:], O.rhs_known(sp, U_start, f))
    R = torch.empty((p.Ns,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-10,
                                                 kernel_flags=flags)) as plan:
        plan.timing_enable(True)
        plan.residual(dev(u0), dev(f), dev(U), R)
        cls = _counts(plan)
    assert cls["dst_tc"]["count"] > 0 and cls["dst"]["count"] == 0, cls
    assert relmax(host(R), ref) < 1e-9


@pytest.mark.parametrize("flags", TILES, ids=["n128", "n64"])
@pytest.mark.parametrize("p", TC_CASES, ids=TC_IDS)
def test_tc_solve_matches_sequential(expd, p, flags):
    sp = O.spec_of(p)
    rng = np.random.default_rng(14)
    u0 = rng.uniform(-0.8, 0.8, p.n)
    f = rng.standard_normal((p.Nt,) + p.n) if p.nonlin == "none" else None
    ref = O.sequential_solve(sp, u0, f)[1:]
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-10, max_iter=200,
                                                 kernel_flags=flags)) as plan:
        info = plan.solve_fp(dev(u0), None if f is None else dev(f), U)
    assert O.rel_error(host(U), ref) < 1e-9, info
    if p.nonlin == "none":
        U2 = torch.empty_like(U)
        with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-10,
                                                     kernel_flags=flags)) as plan:
            info = plan.solve_gmres(dev(u0), dev(f), U2)
        assert O.rel_error(host(U2), ref) < 1e-9, info


def test_tc_agrees_with_float64_products(expd, monkeypatch):
    # the same mixed solve with the float64 dense products (EXPD_DST_TC=0)
    p = TC_CASES[1]
    rng = np.random.default_rng(15)
    u0 = rng.uniform(-0.8, 0.8, p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("EXPD_DST_TC", mode)
        U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
        with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-11)) as plan:
            plan.timing_enable(True)
            plan.solve_gmres(dev(u0), dev(f), U)
            cls = _counts(plan)
        assert (cls["dst_tc"]["count"] > 0) == (mode == "1"), cls
        out[mode] = host(U)
    assert O.rel_error(out["1"], out["0"]) < 1e-9


def test_tc_folded_products_agree_with_full_ones(expd, monkeypatch):
    # S[j][n-1-k] = (-1)^j S[j][k]: the folded transform (half the digit
    # products) and the full one agree to the digits' accuracy
    p = TC_CASES[1]
    r = np.random.default_rng(17).standard_normal((p.Ns,) + p.n)
    out = {}
    for fold in ("1", "0"):
        monkeypatch.setenv("EXPD_DST_FOLD", fold)
        S = torch.empty_like(dev(r))
        with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-10)) as plan:
            plan.timing_enable(True)
            plan.precond_apply(dev(r), S)
            cls = _counts(plan)
        out[fold] = (host(S), cls["dst_tc"]["flops"])
    assert relmax(out["1"][0], out["0"][0]) < 1e-9
    assert out["1"][1] == pytest.approx(out["0"][1] / 2)


def test_tc_tile_widths_agree_bit_for_bit(expd):
    # both tile widths sum the same digit products in the same order per
    # output element: identical results
    p = TC_CASES[1]
    rng = np.random.default_rng(16)
    r = rng.standard_normal((p.Ns,) + p.n)
    out = []
    for flags in TILES:
        S = torch.empty_like(dev(r))
        with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-10,
                                                     kernel_flags=flags)) as plan:
            plan.precond_apply(dev(r), S)
        out.append(host(S))
    assert np.array_equal(out[0], out[1])


def test_tc_deterministic(expd):
    p = TC_CASES[0]
    rng = np.random.default_rng(16)
    u0 = rng.uniform(-1, 1, p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    res = []
    with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-10)) as plan:
        for _ in range(2):
            U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
            plan.solve_fp(dev(u0), dev(f), U)
            res.append(host(U))
    assert np.array_equal(res[0], res[1])


def test_tc_heat_dirichlet_1024_full_mixed_gmres(expd):
    # the 1024^2 Dirichlet heat workload (s = 2, Nt = 128, GMRES, tol 1e-9) on
    # the mixed path: every spatial transform on the tensor cores
    p = I.HEAT_DIRICHLET_1024
    u0, f = I.make_inputs(p)
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED, max_iter=200)) as plan:
        plan.timing_enable(True)
        info = plan.solve_gmres(dev(u0), dev(f), U)
        cls = _counts(plan)
    assert cls["dst_tc"]["count"] > 0 and cls["dst"]["count"] == 0, cls
    ref = O.sequential_solve(O.spec_of(p), u0, f)[1:]
    assert O.rel_error(host(U), ref) < p.tol, info


def test_tc_cancel_in_flight_gives_up_waits_and_gpu_stays_usable(expd):
    # Failure detection without a GPU fault: a cancel request set before the
    # solve makes the tensor-core kernel's pipeline waits give up at once (the
    # kernel waits, with a limit, for its own copies and MMAs, frees TMEM and
    # records the give-up); the call returns EXPD_ERR_CANCELLED, and the next
    # solve on the same plan runs normally and matches the oracle.
    p = TC_CASES[1]
    sp = O.spec_of(p)
    rng = np.random.default_rng(17)
    u0 = rng.standard_normal(p.n)
    f = rng.standard_normal((p.Nt,) + p.n)
    ref = O.sequential_solve(sp, u0, f)[1:]
    U = torch.empty((p.Nt,) + p.n, dtype=torch.float64, device=DEV)
    with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-10, max_iter=100)) as plan:
        plan.timing_enable(True)
        plan.cancel()
        with pytest.raises(expd.ExpdError) as ei:
            plan.solve_gmres(dev(u0), dev(f), U)
        assert ei.value.status == expd.ERR_CANCELLED
        assert _counts(plan)["dst_tc"]["count"] > 0
        plan.solve_gmres(dev(u0), dev(f), U)
        assert _counts(plan)["dst_tc"]["count"] > 0
    assert O.rel_error(host(U), ref) < 1e-9


def test_tc_half_tile_operand_rows_same_bits_every_run(expd):
    # S's folded halves of 192 rows end in a half-filled 128-row tile; each
    # digit slice spans whole tiles, so no digit's tiles overlap the next
    # one's and repeated transforms give the same bits (and the oracle's values)
    p = TC_CASES[-1]
    r = np.random.default_rng(19).standard_normal((p.Ns,) + p.n)
    ref = O.precond_apply(O.spec_of(p), r)
    outs = []
    for _ in range(3):
        S = torch.empty_like(dev(r))
        with expd.plan_create(expd.spec_from_problem(p, precision=expd.PREC_MIXED, tol=1e-10)) as plan:
            plan.precond_apply(dev(r), S)
        outs.append(host(S))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    assert relmax(outs[0], ref) < 6e-8 * 16 / p.alpha
