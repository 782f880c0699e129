"""Error paths of the shifted COCG on the GPU, driven without a GPU fault.

* An expired bounded wait: the solve option wait_cap = -1 gives every CTA's first wait on its TMA
  transfers no attempts, so the wait is declared lost at once.  The CTA raises the device error
  flag, drains every transfer it issued (those waits keep their full cap, so nothing is left in
  flight when the CTA returns) and returns; the host turns the flag into RSFD_ERR_TIMEOUT.  The same
  handle then solves normally and matches the oracle.
* A breakdown (reading 5 of the paper's Appendix: a quasi-null (r_n, r_n)): with breakdown_tol
  raised above any |(r, r)| / ||r||^2, the scalar step reports every column as broken down at its
  first iteration; the status travels through the slot state into rsfd_col_info and the return
  value, the columns' G0_bb stays zero (x_0 = 0), and the next normal solve is unaffected.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from workloads import small_problem                        # noqa: E402
from oracle.cocg import shifted_cocg_columns               # noqa: E402


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_00081_gb300.build_lib import build
    build()
    import paper_1502_00081_gb300 as m
    m.load_library()
    return m


def _problem():
    return small_problem(grid=(20, 12, 16), h=0.45, fd_order=4, n_wells=3, n_energies=4, e_range=(0.3, 2.0),
                         eta=5e-2, tol=1e-10, cols=3)


def _relf(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _solve(rs, h, p, G0):
    st, info, res = rs.rsfd_shifted_cocg(h.ptr, p.cols, p.energies, p.eta, p.tol, p.maxit, G0)
    torch.cuda.synchronize()
    return st, info, G0.cpu().numpy().astype(np.complex128).transpose(0, 2, 1)


@pytest.mark.parametrize("prec,kind", [("FP64", 1), ("FP64", 2), ("DF64", 2)])
def test_expired_wait_reports_timeout_and_handle_recovers(rs, prec, kind):
    p = _problem()
    Go, _ = shifted_cocg_columns(p)
    bound = 1e-9 if prec == "FP64" else 1e-6
    with rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=getattr(rs, "RSFD_" + prec)) as h:
        G0 = torch.zeros((p.K, p.cols.size, h.nb), dtype=h.complex_dtype, device="cuda")
        rs.rsfd_set_solve_options(h.ptr, pass_kind=kind, slots=3, wait_cap=-1)
        with pytest.raises(rs.RsfdError) as e:
            _solve(rs, h, p, G0)
        assert e.value.status == rs.RSFD_ERR_TIMEOUT, e.value
        assert "bounded wait" in str(e.value)
        # the context is intact: a normal solve on the same handle gives the oracle's answer
        rs.rsfd_set_solve_options(h.ptr, pass_kind=kind, slots=3)
        st, info, G = _solve(rs, h, p, G0)
        assert st == rs.RSFD_OK
        assert _relf(G, Go) <= bound


@pytest.mark.parametrize("prec", ["FP64", "DF64"])
def test_breakdown_status_reaches_column_info(rs, prec):
    p = _problem()
    with rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=getattr(rs, "RSFD_" + prec)) as h:
        G0 = torch.full((p.K, p.cols.size, h.nb), 7.0, dtype=h.complex_dtype, device="cuda")
        rs.rsfd_set_solve_options(h.ptr, slots=2, breakdown_tol=1e300)
        st, info, G = _solve(rs, h, p, G0)
        assert st == rs.RSFD_ERR_BREAKDOWN
        assert (info["status"] == rs.RSFD_ERR_BREAKDOWN).all()
        assert (info["iters"] == 0).all()
        assert "breakdown" in rs.rsfd_last_error(h.ptr)
        assert np.all(G == 0)          # x_0 = 0 is what a column that broke down at once holds
        rs.rsfd_set_solve_options(h.ptr, slots=2)
        st, info, G = _solve(rs, h, p, G0)
        assert st == rs.RSFD_OK and (info["status"] == 0).all()
        Go, _ = shifted_cocg_columns(p)
        assert _relf(G, Go) <= (1e-9 if prec == "FP64" else 1e-6)
