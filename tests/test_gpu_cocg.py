"""GPU parity of the shifted COCG path (Sec. III B, Appendix) against the CPU oracle.

All calls go through the C ABI (ctypes binding).  FP64 mode must match the oracle to a relative
Frobenius error <= 1e-9; mixed mode (complex64 vectors, FP64 scalars and reductions) is compared
with a bound derived from single precision (see the individual tests).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from workloads import make_problem, small_problem          # noqa: E402
from oracle.cocg import shifted_cocg_columns               # noqa: E402
from oracle.operator import boundary_rows                  # noqa: E402
from oracle.dense import g0_dense                          # noqa: E402


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_00081_gb300.build_lib import build
    build()
    import paper_1502_00081_gb300 as m
    m.load_library()
    return m


def gpu_g0(rs, p, precision, cols=None, opts=None, seed_kind=0, seed_index=0, tol=None, maxit=None):
    cols = p.cols if cols is None else np.asarray(cols)
    with rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=precision) as h:
        if opts:
            rs.rsfd_set_solve_options(h.ptr, **opts)
        G0 = torch.zeros((p.K, cols.size, h.nb), dtype=h.complex_dtype, device="cuda")
        st, info, res = rs.rsfd_shifted_cocg(h.ptr, cols, p.energies, p.eta, p.tol if tol is None else tol,
                                             p.maxit if maxit is None else maxit, G0, seed_kind, seed_index)
        stats = rs.rsfd_get_stats(h.ptr)
        torch.cuda.synchronize()
        out = G0.cpu().numpy().astype(np.complex128).transpose(0, 2, 1)   # [K, nb, ncols]
    return st, out, info, res, stats


def relf(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


KINDS = [1, 2, 3]   # RSFD_PASS_RECOMPUTE (fused, three vectors), RSFD_PASS_STORED (five vectors), RSFD_PASS_SPLIT
                    # (the five-vector iteration as a combine launch and a stencil launch)


@pytest.mark.parametrize("kind", KINDS)
def test_tiny_wire_fp64_matches_oracle_and_dense(rs, kind):
    """The 8x8x12 2nd-order wire, all 128 plane columns, 8 energies, tol 1e-12."""
    p = make_problem("tiny_wire_fp64")
    st, G, info, res, stats = gpu_g0(rs, p, rs.RSFD_FP64, opts=dict(pass_kind=kind))
    assert st == rs.RSFD_OK
    b = boundary_rows(p.grid, p.n_face)
    Go, ores = shifted_cocg_columns(p)
    assert relf(G, Go) <= 1e-9
    for k in (0, 3, 7):
        Gd = g0_dense(p, p.energies[k] + 1j * p.eta, rows=b, cols=p.cols)
        assert relf(G[k], Gd) <= 1e-9
    # complex symmetry of the boundary block (rows == cols here)
    assert np.abs(G - G.transpose(0, 2, 1)).max() <= 1e-9 * np.abs(G).max()
    assert (info["status"] == 0).all() and (res < p.tol).all()
    # iteration counts agree with the oracle's to within rounding-order noise: the stopping iteration
    # is where ||r_n|| / |pi_n| (Eq. collinear) crosses 1e-12, and the oracle itself moves individual
    # columns by up to ~5 iterations when only the summation order of its dots changes
    it_o = np.array([r.iterations for r in ores])
    assert np.abs(info["iters"] - it_o).max() <= 8
    assert abs(float(np.mean(info["iters"] - it_o))) <= 3


@pytest.mark.parametrize("grid,order,slots,tile_y,zc", [
    ((37, 13, 45), 4, 3, 8, 16),     # ragged x, y and z tiles, slot refill
    ((9, 33, 20), 2, 2, 12, 7),
    ((5, 4, 6), 4, 8, 0, 0),         # tiles far larger than the grid
])
@pytest.mark.parametrize("kind", KINDS)
def test_ragged_tiles_fp64(rs, grid, order, slots, tile_y, zc, kind):
    p = small_problem(grid=grid, h=0.45, fd_order=order, n_wells=4, n_energies=5, e_range=(0.3, 2.5),
                      eta=5e-2, tol=1e-12, cols=7)
    st, G, info, res, _ = gpu_g0(rs, p, rs.RSFD_FP64,
                                 opts=dict(slots=slots, tile_y=tile_y, z_chunk=zc, pass_kind=kind))
    assert st == rs.RSFD_OK
    Go, _ = shifted_cocg_columns(p)
    assert relf(G, Go) <= 1e-9


@pytest.mark.parametrize("pkind", KINDS)
def test_seed_switching_and_policies(rs, pkind):
    """Seed switches (Eq. seedswitch); in the stored-product pass the switch also moves the stored
    A r_n to the new seed energy, which a wrong shift would put into every later iterate."""
    p = small_problem(grid=(7, 6, 12), h=0.5, fd_order=4, n_wells=3, n_energies=6, e_range=(-4.0, 3.0),
                      eta=2e-2, tol=1e-12, cols=4)
    Go, ores = shifted_cocg_columns(p, seed=0)
    assert max(r.switches for r in ores) >= 1
    for kind, idx in ((rs.RSFD_SEED_FIRST, 0), (rs.RSFD_SEED_MID, 0), (rs.RSFD_SEED_INDEX, 5)):
        st, G, info, res, _ = gpu_g0(rs, p, rs.RSFD_FP64, seed_kind=kind, seed_index=idx,
                                     opts=dict(pass_kind=pkind))
        assert st == rs.RSFD_OK
        assert relf(G, Go) <= 1e-9
        if kind == rs.RSFD_SEED_FIRST:
            assert info["switches"].max() >= 1


@pytest.mark.parametrize("prec,kind", [("DF64", 2), ("DF64", 1), ("DF64", 3), ("MIXED", 1), ("MIXED", 2), ("MIXED", 3)])
def test_launch_modes_bitwise_identical(rs, prec, kind):
    """Graph replay, plain launches, profiled launches and another collapse length all run the same
    fixed-order reductions; the collapse length only regroups exact-order sums of the shift update,
    so it is compared with a tolerance instead."""
    p = small_problem(grid=(16, 12, 20), h=0.45, fd_order=4, n_wells=3, n_energies=4, e_range=(0.2, 2.0),
                      eta=3e-2, tol=1e-6 if prec == "DF64" else 1e-5, cols=6)
    outs = []
    for opts in (dict(slots=3), dict(slots=3, use_graphs=-1), dict(slots=3, profile=1)):
        opts["pass_kind"] = kind
        st, G, info, res, stats = gpu_g0(rs, p, getattr(rs, "RSFD_" + prec), opts=opts)
        assert st == rs.RSFD_OK
        outs.append(G)
        if opts.get("profile"):
            assert stats["ms_pass"] > 0 and stats["ms_shift"] > 0
    for G in outs[1:]:
        assert np.array_equal(G, outs[0])
    st, G5, info, res, stats = gpu_g0(rs, p, getattr(rs, "RSFD_" + prec),
                                      opts=dict(slots=3, iters_per_sync=5, pass_kind=kind))
    assert st == rs.RSFD_OK
    assert relf(G5, outs[0]) <= 1e-5


@pytest.mark.parametrize("kind", KINDS)
def test_double_float_matches_oracle_at_small_eta(rs, kind):
    """Double-float vectors (RSFD_DF64) on a grid and eta where complex64 Krylov vectors stall: the
    error is set by the FP32 contributions of the collapsed shift update (about 1e-7), far inside
    the stated mixed-mode tolerance."""
    p = small_problem(grid=(24, 24, 40), h=0.4, fd_order=4, n_wells=8, n_energies=8, e_range=(-0.5, 0.5),
                      eta=1e-3, tol=1e-8, cols=3)
    st, G, info, res, _ = gpu_g0(rs, p, rs.RSFD_DF64, opts=dict(pass_kind=kind))
    assert st == rs.RSFD_OK
    Go, ores = shifted_cocg_columns(p, tol=1e-11)
    err = relf(G, Go)
    assert err <= 1e-6, err
    # iteration counts stay close to the FP64 oracle's
    it_o = np.array([r.iterations for r in ores])
    assert (info["iters"] <= 1.3 * it_o + 50).all()


@pytest.mark.parametrize("kind", KINDS)
def test_mixed_precision_matches_oracle(rs, kind):
    """complex64 Krylov vectors with FP64 scalars.  The error of G0 is set by the gap between the
    recursive and the true residual that single-precision storage of r_n opens (about
    eps_32 * sum_k ||r_k|| per unit right-hand side, amplified by ||(Z - H)^{-1}|| <= 1/eta); a CPU
    simulation of the same arithmetic gives 0.5-2.5e-5 on grids of this size, so the bound is 5e-5.
    (The stated mixed-mode tolerance, 1e-5, applies to G_bb; see test_gpu_dyson_T.)"""
    p = small_problem(grid=(24, 20, 32), h=0.4, fd_order=4, n_wells=6, n_energies=8, e_range=(-0.5, 0.5),
                      eta=1e-2, tol=1e-7, cols=6)
    st, G, info, res, _ = gpu_g0(rs, p, rs.RSFD_MIXED, opts=dict(pass_kind=kind))
    assert st == rs.RSFD_OK
    Go, _ = shifted_cocg_columns(p, tol=1e-12)
    err = relf(G, Go)
    assert err <= 5e-5, err


def test_maxit_reports_not_converged(rs):
    p = small_problem(grid=(8, 8, 12), h=0.5, fd_order=2, n_wells=2, n_energies=3, eta=1e-3, tol=1e-12, cols=2)
    st, G, info, res, _ = gpu_g0(rs, p, rs.RSFD_FP64, maxit=5)
    assert st == rs.RSFD_ERR_NOT_CONVERGED
    assert (info["iters"] == 5).all() and (info["status"] == rs.RSFD_ERR_NOT_CONVERGED).all()


def test_argument_errors(rs):
    p = small_problem(grid=(6, 5, 8), cols=2)
    with rs.Handle(p.grid, p.h, p.fd_order, p.V) as h:
        G0 = torch.zeros((p.K, 2, h.nb), dtype=torch.complex128, device="cuda")
        for bad in (dict(cols=np.array([-1, 3])), dict(eta=0.0), dict(tol=2.0)):
            args = dict(cols=p.cols, eta=p.eta, tol=p.tol)
            args.update(bad)
            with pytest.raises(rs.RsfdError):
                rs.rsfd_shifted_cocg(h.ptr, args["cols"], p.energies, args["eta"], args["tol"], 100, G0)
        # launch options the pass cannot honour are rejected before any launch
        for bad in (dict(pass_kind=5), dict(rows_per_thread=3), dict(prefetch=8), dict(pass_kind=2, tile_y=6,
                                                                                   rows_per_thread=4),
                    dict(pass_kind=2, tile_y=64)):
            with pytest.raises(rs.RsfdError):
                rs.rsfd_set_solve_options(h.ptr, **bad)


@pytest.mark.parametrize("rows,tile_y", [(1, 8), (2, 12), (4, 8)])
def test_stored_pass_rows_per_thread(rs, rows, tile_y):
    """Every thread organisation of the stored-product pass (tile rows per thread, ragged tiles in x,
    y and z) gives the oracle's G0 in FP64."""
    p = small_problem(grid=(37, 26, 19), h=0.45, fd_order=4, n_wells=4, n_energies=5, e_range=(0.3, 2.5),
                      eta=5e-2, tol=1e-12, cols=5)
    st, G, info, res, _ = gpu_g0(rs, p, rs.RSFD_FP64, opts=dict(pass_kind=2, rows_per_thread=rows, tile_y=tile_y,
                                                                  slots=3, z_chunk=7))
    assert st == rs.RSFD_OK
    Go, _ = shifted_cocg_columns(p)
    assert relf(G, Go) <= 1e-9


@pytest.mark.parametrize("tile_y", [8, 12, 14])
def test_double_float_register_budget_variant_identical(rs, tile_y):
    """The 128-register variant of the one-row double-float stored pass (one CTA per SM, no spills)
    computes exactly what the 96-register variant computes (same arithmetic, bit for bit), on ragged
    tiles in x, y and z with seed switching."""
    p = small_problem(grid=(45, 30, 21), h=0.45, fd_order=4, n_wells=4, n_energies=6, e_range=(0.3, 2.5),
                      eta=4e-2, tol=1e-9, cols=4)
    outs = []
    for budget in (0, 1):
        st, G, info, res, _ = gpu_g0(rs, p, rs.RSFD_DF64, opts=dict(pass_kind=2, rows_per_thread=1, tile_y=tile_y,
                                                                      slots=3, z_chunk=9, reg_budget=budget))
        assert st == rs.RSFD_OK
        outs.append((G, info["iters"].copy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    Go, _ = shifted_cocg_columns(p, tol=1e-11)
    assert relf(outs[1][0], Go) <= 1e-6


@pytest.mark.parametrize("grid,order,tile_y", [((48, 26, 19), 4, 8), ((40, 30, 17), 4, 14), ((48, 20, 15), 2, 16)])
def test_double_float_sixteen_wide_tiles(rs, grid, order, tile_y):
    """The 16-wide tile of the one-row double-float stored pass (two tile rows per warp), on grids whose
    width is an odd multiple of 16 or ragged, against the oracle; the 32-wide tile (another summation
    order of the dot products) agrees with it within the double-float error (~1e-7, the FP32 leading
    parts of the recorded residual rows)."""
    p = small_problem(grid=grid, h=0.45, fd_order=order, n_wells=4, n_energies=6, e_range=(0.3, 2.5),
                      eta=4e-2, tol=1e-10, cols=4)
    outs = []
    for tx in (16, 32):
        st, G, info, res, _ = gpu_g0(rs, p, rs.RSFD_DF64, opts=dict(pass_kind=2, rows_per_thread=1, tile_y=tile_y,
                                                                      slots=3, z_chunk=7, tile_x=tx))
        assert st == rs.RSFD_OK
        outs.append((G, info["iters"].copy()))
    Go, _ = shifted_cocg_columns(p, tol=1e-12)
    assert relf(outs[0][0], Go) <= 1e-6
    assert relf(outs[0][0], outs[1][0]) <= 1e-6
    # near the double-float floor the iteration count follows the rounding of the dots (a few per cent)
    assert (np.abs(outs[0][1] - outs[1][1]) <= 0.05 * outs[1][1]).all()


@pytest.mark.parametrize("grid", [(64, 18, 16), (40, 20, 18)])
def test_double_float_bench_shape_fourth_order(rs, grid):
    """The launch shape of the benchmarked 64x64x128 run (stored pass, 32 x 16 tile, one row per thread,
    the whole z extent per CTA, 96-register variant) on a 4th-order (R = 2) grid with seed switching:
    full x tiles and ragged x, y tiles, against the FP64 oracle."""
    p = small_problem(grid=grid, h=0.4, fd_order=4, n_wells=6, n_energies=6, e_range=(-0.5, 0.5),
                      eta=5e-2, tol=1e-10, cols=2, n_face=1)
    opts = dict(pass_kind=2, tile_y=16, rows_per_thread=1, z_chunk=grid[2], tile_x=32, reg_budget=0, slots=2)
    st, G, info, res, _ = gpu_g0(rs, p, rs.RSFD_DF64, opts=opts)
    assert st == rs.RSFD_OK
    Go, ores = shifted_cocg_columns(p, tol=1e-12)
    assert relf(G, Go) <= 1e-6
    assert max(r.switches for r in ores) >= 1


@pytest.mark.parametrize("prec,bound", [("FP64", 1e-9), ("DF64", 1e-6)])
def test_seed_outside_the_energy_set(rs, prec, bound):
    """Auxiliary seed energies (the extension of Eq. seedswitch to an energy outside the set): the
    first seed far below the spectrum, and a switch target inside it, against the oracle run with the
    same auxiliary energies and against the oracle with an in-set seed."""
    from oracle.cocg import shifted_cocg
    from oracle.operator import hamiltonian, apply_h
    p = small_problem(grid=(12, 10, 14), h=0.5, fd_order=4, n_wells=2, n_energies=5, e_range=(-3.0, -1.0),
                      eta=5e-2, tol=1e-11, cols=3)
    H, P, wE = hamiltonian(p)
    b_rows = boundary_rows(p.grid, p.n_face)
    Z = p.energies + 1j * p.eta
    aux = np.array([-12.0, 1.7])
    cases = [(rs.RSFD_SEED_AUX, 0, ("aux", 0)), (rs.RSFD_SEED_FIRST, 0, "first")]
    Gref, _ = shifted_cocg_columns(p, tol=1e-12)
    for kind, idx, oseed in cases:
        Go = np.zeros((p.K, b_rows.size, p.cols.size), complex)
        osw = []
        for jj, j in enumerate(p.cols):
            b = np.zeros(p.N, complex)
            b[j] = 1.0
            r = shifted_cocg(lambda v: apply_h(H, P, wE, v), b, Z, p.tol, rows=b_rows, seed=oseed,
                             aux=aux + 1j * p.eta)
            Go[:, :, jj] = r.x
            osw.append(r.seeds[-1])
        with rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=getattr(rs, "RSFD_" + prec)) as h:
            G0 = torch.zeros((p.K, p.cols.size, h.nb), dtype=h.complex_dtype, device="cuda")
            st, info, res = rs.rsfd_shifted_cocg(h.ptr, p.cols, p.energies, p.eta, p.tol, p.maxit, G0, kind, idx,
                                                 aux_energies=aux)
            torch.cuda.synchronize()
            G = G0.cpu().numpy().astype(np.complex128).transpose(0, 2, 1)
        assert st == rs.RSFD_OK and res.shape == (p.cols.size, p.K)
        # the seed ends on the auxiliary energy inside the spectrum (index K + 1), as in the oracle
        assert (info["switches"] >= 1).all() and list(info["final_seed"]) == osw == [p.K + 1] * p.cols.size
        assert relf(G, Go) <= bound
        assert relf(G, Gref) <= max(bound, 1e-9)


BFP_CASES = [((64, 18, 16), 4, 16, 16), ((40, 30, 17), 4, 8, 7), ((37, 26, 19), 4, 4, 19), ((48, 20, 15), 2, 16, 8),
             ((33, 17, 13), 2, 8, 13)]


@pytest.mark.parametrize("grid,order,tile_y,z_chunk", BFP_CASES)
def test_block_floating_point_split_pass(rs, grid, order, tile_y, z_chunk):
    """RSFD_PASS_SPLIT_BFP (leading parts of r_n on a per-column quantum, the product stored as s A r
    with integer neighbour weights) on full and ragged tiles in x, y and z, 2nd and 4th order, with
    seed switching: against the FP64 oracle, and against the plain split pass (the same iteration up
    to double-float rounding: equal G0 within the double-float error, iteration counts within a few
    per cent)."""
    p = small_problem(grid=grid, h=0.4, fd_order=order, n_wells=6, n_energies=6, e_range=(-0.5, 0.5),
                      eta=5e-2, tol=1e-10, cols=3, n_face=1)
    outs = {}
    for kind in (3, 4):
        st, G, info, res, stats = gpu_g0(rs, p, rs.RSFD_DF64, opts=dict(pass_kind=kind, tile_y=tile_y,
                                                                          z_chunk=z_chunk, slots=2))
        assert st == rs.RSFD_OK
        outs[kind] = (G, info["iters"].copy(), res)
    Go, ores = shifted_cocg_columns(p, tol=1e-12)
    assert max(r.switches for r in ores) >= 1
    assert relf(outs[4][0], Go) <= 1e-6
    assert relf(outs[4][0], outs[3][0]) <= 1e-6
    assert (np.abs(outs[4][1] - outs[3][1]) <= 0.12 * outs[3][1] + 2).all()
    assert (outs[4][2] < p.tol).all()


def test_block_floating_point_kind_resolves_elsewhere(rs):
    """FP64 and complex64 handles run the plain split pass when asked for the block-floating-point
    form: bit-identical results."""
    p = small_problem(grid=(24, 14, 12), h=0.45, fd_order=4, n_wells=3, n_energies=4, e_range=(0.3, 2.0),
                      eta=5e-2, tol=1e-10, cols=3)
    for prec in (rs.RSFD_FP64, rs.RSFD_MIXED):
        a = gpu_g0(rs, p, prec, opts=dict(pass_kind=3, slots=2), tol=1e-5 if prec == rs.RSFD_MIXED else None)
        b = gpu_g0(rs, p, prec, opts=dict(pass_kind=4, slots=2), tol=1e-5 if prec == rs.RSFD_MIXED else None)
        assert a[0] == b[0] == rs.RSFD_OK
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2]["iters"], b[2]["iters"])
