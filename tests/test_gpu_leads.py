"""GPU parity of the lead self-energies by decimation (Eq. self-energy with the surface Green's
function of Eq. surface green's function) for leads that repeat one principal layer with its own
potential, against the oracle: the Bloch-root closed form at V = 0 and the oracle's decimation with the
same layer potentials; then Dyson and T with such leads against the oracle's."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from workloads import small_problem                                   # noqa: E402
from oracle.leads import sigma_bloch, sigma_sancho_rubio              # noqa: E402
from oracle.cocg import shifted_cocg_columns                          # noqa: E402
from oracle.operator import boundary_rows                             # noqa: E402
from oracle.dyson import dyson_solve                                  # noqa: E402
from oracle.transmission import transmission                          # noqa: E402


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_00081_gb300.build_lib import build
    build()
    import paper_1502_00081_gb300 as m
    m.load_library()
    return m


def _mats(t):
    return t.cpu().numpy().transpose(0, 2, 1)   # column-major device layout -> [K, rows, cols]


@pytest.mark.parametrize("order,nx,ny", [(2, 5, 4), (4, 4, 3), (4, 7, 6)])
def test_decimation_uniform_lead_matches_closed_form(rs, order, nx, ny):
    R = order // 2
    E = np.array([0.4, 1.1, 2.7, 5.0])
    eta = 1e-2
    with rs.Handle((nx, ny, 2 * R + 2), 0.5, order, np.zeros(nx * ny * (2 * R + 2)), precision=rs.RSFD_FP64) as h:
        SL, SR, it = rs.rsfd_lead_sigma_decimation(h.ptr, E, eta)
        SLg, SRg = _mats(SL), _mats(SR)
    assert 1 <= it < 200
    for k, e in enumerate(E):
        SLo, SRo = sigma_bloch(nx, ny, 0.5, order, e + 1j * eta)
        assert np.abs(SLg[k] - SLo).max() <= 1e-9 * np.abs(SLo).max()
        assert np.abs(SRg[k] - SRo).max() <= 1e-9 * np.abs(SRo).max()


@pytest.mark.parametrize("order", [2, 4])
def test_decimation_periodic_leads_match_oracle(rs, order):
    R = order // 2
    nx, ny = 5, 4
    rng = np.random.Generator(np.random.PCG64(9))
    VL = rng.uniform(-0.8, 0.3, size=(R, ny, nx))
    VR = rng.uniform(-0.8, 0.3, size=(R, ny, nx))
    E, eta = np.array([0.3, 0.9, 1.7]), 5e-3
    with rs.Handle((nx, ny, 2 * R + 2), 0.5, order, np.zeros(nx * ny * (2 * R + 2)), precision=rs.RSFD_FP64) as h:
        SL, SR, it = rs.rsfd_lead_sigma_decimation(h.ptr, E, eta, V_left=VL, V_right=VR)
        SLg, SRg = _mats(SL), _mats(SR)
    for k, e in enumerate(E):
        SLo, SRo = sigma_sancho_rubio(nx, ny, 0.5, order, e + 1j * eta, V_left=VL, V_right=VR)
        assert np.abs(SLg[k] - SLo).max() <= 1e-9 * np.abs(SLo).max()
        assert np.abs(SRg[k] - SRo).max() <= 1e-9 * np.abs(SRo).max()


def test_wire_with_periodic_leads_dyson_and_T(rs):
    """G0_bb (GPU shifted COCG) -> Sigma by GPU decimation for leads with their own potentials ->
    Dyson -> T, against the oracle's G0_bb, decimated Sigma, Dyson solve and T."""
    p = small_problem(grid=(6, 5, 12), h=0.5, fd_order=4, n_wells=2, n_energies=4, e_range=(0.6, 2.2),
                      eta=2e-2, tol=1e-12)
    rng = np.random.Generator(np.random.PCG64(12))
    VL = rng.uniform(-0.5, 0.0, size=(2, 5, 6))
    VR = rng.uniform(-0.5, 0.0, size=(2, 5, 6))
    b = boundary_rows(p.grid, p.n_face)
    with rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=rs.RSFD_FP64) as h:
        G0 = torch.zeros((p.K, h.nb, h.nb), dtype=torch.complex128, device="cuda")
        st, info, res = rs.rsfd_shifted_cocg(h.ptr, h.rows, p.energies, p.eta, p.tol, p.maxit, G0)
        assert st == rs.RSFD_OK
        SL, SR, it = rs.rsfd_lead_sigma_decimation(h.ptr, p.energies, p.eta, V_left=VL, V_right=VR)
        G = torch.empty_like(G0)
        rs.rsfd_dyson_boundary(h.ptr, G0, SL, SR, G)
        T = rs.rsfd_transmission(h.ptr, G, SL, SR)
    G0o, _ = shifted_cocg_columns(p, cols=b, rows=b, tol=1e-13)
    for k, E in enumerate(p.energies):
        SLo, SRo = sigma_sancho_rubio(p.grid[0], p.grid[1], p.h, p.fd_order, E + 1j * p.eta, V_left=VL, V_right=VR)
        To = transmission(dyson_solve(G0o[k], SLo, SRo), SLo, SRo)[0]
        assert abs(T[k] - To) <= 1e-8 * max(1.0, abs(To))
