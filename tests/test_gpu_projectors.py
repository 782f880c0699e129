"""GPU parity of the nonlocal projector term of the seed SpMV (separable Kleinman-Bylander
projectors, Sec. II A: V_nl psi = sum_a E_a p_a (p_a^T psi) h^3) inside the shifted COCG of
Sec. III B, against the CPU oracle: dense (Z - H_T)^{-1} on small grids, the oracle's own shifted
COCG iterates on ragged multi-tile grids and on the full 72 x 72 x 256 peapod-shaped grid with its
460 projectors (a fixed number of iterations, sampled columns)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from workloads import make_problem, small_problem   # noqa: E402
from oracle.cocg import shifted_cocg_columns        # noqa: E402
from oracle.operator import boundary_rows           # noqa: E402
from oracle.dense import g0_dense                   # noqa: E402


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_00081_gb300.build_lib import build
    build()
    import paper_1502_00081_gb300 as m
    m.load_library()
    return m


def gpu_g0(rs, p, precision, cols, tol=None, maxit=None, opts=None):
    cols = np.asarray(cols)
    with rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, proj=p.proj, precision=precision) as h:
        if opts:
            rs.rsfd_set_solve_options(h.ptr, **opts)
        G0 = torch.zeros((p.K, cols.size, h.nb), dtype=h.complex_dtype, device="cuda")
        st, info, res = rs.rsfd_shifted_cocg(h.ptr, cols, p.energies, p.eta, p.tol if tol is None else tol,
                                             p.maxit if maxit is None else maxit, G0)
        torch.cuda.synchronize()
        out = G0.cpu().numpy().astype(np.complex128).transpose(0, 2, 1)   # [K, nb, ncols]
    return st, out, info


def relf(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("order", [2, 4])
def test_projectors_fp64_match_dense(rs, order):
    """FP64 handle with 3 projectors: G0_bb equals the dense inverse of Z - H_T (local + nonlocal)."""
    p = small_problem(grid=(8, 7, 12), h=0.5, fd_order=order, n_wells=2, projectors=3, n_energies=4,
                      e_range=(0.3, 1.5), eta=5e-2, tol=1e-12, cols=5)
    assert p.proj is not None and p.proj.n_atoms == 3
    st, G, info = gpu_g0(rs, p, rs.RSFD_FP64, p.cols)
    assert st == rs.RSFD_OK
    b = boundary_rows(p.grid, p.n_face)
    for k in range(p.K):
        Gd = g0_dense(p, p.energies[k] + 1j * p.eta, rows=b, cols=p.cols)
        assert relf(G[k], Gd) <= 1e-9
    # the projector term matters here: without it the answer is far off
    p0 = small_problem(grid=(8, 7, 12), h=0.5, fd_order=order, n_wells=2, projectors=0, n_energies=4,
                       e_range=(0.3, 1.5), eta=5e-2, tol=1e-12, cols=5)
    Gd0 = g0_dense(p0, p.energies[0] + 1j * p.eta, rows=b, cols=p.cols)
    assert relf(G[0], Gd0) > 1e-3


@pytest.mark.parametrize("prec,tol,bound", [("DF64", 1e-10, 1e-6), ("MIXED", 1e-6, 2e-4)])
def test_projectors_reduced_precision_match_dense(rs, prec, tol, bound):
    """Double-float and complex64 handles with 4 projectors.  Double-float: the error is set by the
    FP32 leading parts of the recorded residual rows that feed the collapsed shift update (~1e-7)."""
    p = small_problem(grid=(9, 8, 14), h=0.45, fd_order=4, n_wells=2, projectors=4, n_energies=5,
                      e_range=(0.5, 2.0), eta=1e-1, tol=tol, cols=4)
    st, G, info = gpu_g0(rs, p, getattr(rs, "RSFD_" + prec), p.cols)
    assert st == rs.RSFD_OK
    b = boundary_rows(p.grid, p.n_face)
    for k in range(p.K):
        Gd = g0_dense(p, p.energies[k] + 1j * p.eta, rows=b, cols=p.cols)
        assert relf(G[k], Gd) <= bound


@pytest.mark.parametrize("kind", [2, 3])
@pytest.mark.parametrize("grid,slots,tile_y", [((37, 21, 20), 3, 8), ((40, 18, 17), 5, 16)])
def test_projectors_ragged_tiles_match_oracle(rs, grid, slots, tile_y, kind):
    """Several x/y tiles with ragged edges, overlapping projector supports, seed switching: the GPU
    iterates equal the oracle's shifted COCG (FP64)."""
    p = small_problem(grid=grid, h=0.5, fd_order=4, n_wells=3, projectors=6, n_energies=5,
                      e_range=(0.5, 2.5), eta=5e-2, tol=1e-11, cols=slots + 2)
    st, G, info = gpu_g0(rs, p, rs.RSFD_FP64, p.cols, opts=dict(slots=slots, tile_y=tile_y, pass_kind=kind))
    assert st == rs.RSFD_OK
    Go, res = shifted_cocg_columns(p, cols=p.cols, tol=1e-11)
    assert relf(G, Go) <= 1e-9
    assert max(r.switches for r in res) >= 1


@pytest.fixture(scope="module")
def peapod_oracle():
    """The peapod-shaped workload, two sampled columns and the oracle's iterates after 40 steps."""
    p = make_problem("peapod")
    cols = p.cols[[0, len(p.cols) // 2 + 7]]
    Go, res = shifted_cocg_columns(p, cols=cols, maxit=40)
    assert all(r.iterations == 40 for r in res)
    return p, cols, Go


@pytest.mark.parametrize("prec,bound,kind", [("FP64", 1e-10, 2), ("DF64", 1e-6, 2), ("DF64", 1e-6, 3),
                                              ("DF64", 1e-6, 4)])
def test_peapod_full_size_first_iterations_match_oracle(rs, peapod_oracle, prec, bound, kind):
    """The 72 x 72 x 256 peapod-shaped workload (460 wells + 460 KB projectors, 100 energies): the
    boundary rows of x^(i) after 40 iterations for two sampled columns equal the oracle's."""
    p, cols, Go = peapod_oracle
    st, G, info = gpu_g0(rs, p, getattr(rs, "RSFD_" + prec), cols, maxit=40, opts=dict(pass_kind=kind))
    assert st == rs.RSFD_ERR_NOT_CONVERGED
    assert (info["iters"] == 40).all()
    assert relf(G, Go) <= bound


@pytest.mark.parametrize("grid,order,tile_y", [((37, 21, 20), 4, 8), ((40, 18, 17), 4, 16), ((33, 20, 16), 2, 8)])
def test_projectors_block_floating_point_pass(rs, grid, order, tile_y):
    """The block-floating-point split pass with projectors (its bound on |s A r| includes the projector
    term: atoms per support point x the largest |s E_a c_a| max|p_a|): ragged tiles, overlapping
    supports, seed switching, against the oracle's converged G0 and the plain split pass."""
    p = small_problem(grid=grid, h=0.45, fd_order=order, n_wells=3, projectors=6, n_energies=5,
                      e_range=(0.5, 2.5), eta=5e-2, tol=1e-10, cols=5)
    outs = {}
    for kind in (3, 4):
        st, G, info = gpu_g0(rs, p, rs.RSFD_DF64, p.cols, opts=dict(slots=3, tile_y=tile_y, pass_kind=kind))
        assert st == rs.RSFD_OK
        outs[kind] = (G, info["iters"].copy())
    Go, res = shifted_cocg_columns(p, cols=p.cols, tol=1e-12)
    assert max(r.switches for r in res) >= 1
    assert relf(outs[4][0], Go) <= 1e-6
    assert relf(outs[4][0], outs[3][0]) <= 1e-6
    assert (np.abs(outs[4][1] - outs[3][1]) <= 0.12 * outs[3][1] + 2).all()
