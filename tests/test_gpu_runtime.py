"""GPU checks of the solver runtime around the shifted COCG of Sec. III B: the launch-option
autotuner (every option it can pick gives the oracle's answer; cached per process) and the
multi-region call (several transition regions of different sizes in one call, results identical to
separate calls and to the oracle)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from workloads import small_problem                 # noqa: E402
from oracle.cocg import shifted_cocg_columns        # noqa: E402


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_00081_gb300.build_lib import build
    build()
    import paper_1502_00081_gb300 as m
    m.load_library()
    return m


def relf(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _solve(rs, h, p, cols, G0):
    st, info, res = rs.rsfd_shifted_cocg(h.ptr, cols, p.energies, p.eta, p.tol, p.maxit, G0)
    torch.cuda.synchronize()
    return st, G0.cpu().numpy().astype(np.complex128).transpose(0, 2, 1), info


@pytest.mark.parametrize("prec", ["FP64", "DF64"])
def test_autotune_options_give_the_oracle_result(rs, prec):
    p = small_problem(grid=(36, 20, 24), h=0.5, fd_order=4, n_wells=3, n_energies=6, e_range=(0.5, 2.0),
                      eta=5e-2, tol=1e-11, cols=5)
    with rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=getattr(rs, "RSFD_" + prec)) as h:
        opts, us = rs.rsfd_autotune(h.ptr, p.energies, p.eta, slots=5, iters=64)
        assert us > 0
        assert opts["pass_kind"] in (rs.RSFD_PASS_RECOMPUTE, rs.RSFD_PASS_STORED, rs.RSFD_PASS_SPLIT,
                                     rs.RSFD_PASS_SPLIT_BFP)
        assert opts["slots"] == 5 and opts["iters_per_sync"] >= 1
        # a second call on the same shape is served from the cache
        opts2, us2 = rs.rsfd_autotune(h.ptr, p.energies, p.eta, slots=5, iters=64)
        assert opts2 == opts and us2 == us
        G0 = torch.zeros((p.K, p.cols.size, h.nb), dtype=h.complex_dtype, device="cuda")
        st, G, info = _solve(rs, h, p, p.cols, G0)
    assert st == rs.RSFD_OK
    Go, _ = shifted_cocg_columns(p, tol=1e-12)
    assert relf(G, Go) <= (1e-9 if prec == "FP64" else 1e-6)


def test_regions_in_one_call_equal_separate_calls(rs):
    """Three regions of different grids, orders and energy sets: one rsfd_shifted_cocg_regions call
    gives bit-for-bit the results of three separate calls, and the oracle's."""
    probs = [small_problem(grid=(12, 10, 16), h=0.5, fd_order=2, n_wells=2, n_energies=4, e_range=(0.4, 1.6),
                           eta=5e-2, tol=1e-12, cols=3, seed=3),
             small_problem(grid=(33, 17, 20), h=0.45, fd_order=4, n_wells=3, n_energies=7, e_range=(0.5, 2.5),
                           eta=4e-2, tol=1e-12, cols=4, seed=4),
             small_problem(grid=(20, 24, 28), h=0.5, fd_order=4, n_wells=2, n_energies=5, e_range=(0.3, 1.8),
                           eta=6e-2, tol=1e-12, cols=2, seed=5)]
    handles = [rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=rs.RSFD_FP64) for p in probs]
    try:
        sep = []
        for p, h in zip(probs, handles):
            G0 = torch.zeros((p.K, p.cols.size, h.nb), dtype=torch.complex128, device="cuda")
            st, G, info = _solve(rs, h, p, p.cols, G0)
            assert st == rs.RSFD_OK
            sep.append(G)
        outs = [torch.zeros((p.K, p.cols.size, h.nb), dtype=torch.complex128, device="cuda")
                for p, h in zip(probs, handles)]
        jobs = [dict(h=h.ptr, cols=p.cols, energies=p.energies, eta=p.eta, tol=p.tol, maxit=p.maxit, G0_bb=o)
                for p, h, o in zip(probs, handles, outs)]
        st, per = rs.rsfd_shifted_cocg_regions(jobs)
        torch.cuda.synchronize()
        assert st == rs.RSFD_OK and all(x[0] == rs.RSFD_OK for x in per)
        for o, G in zip(outs, sep):
            assert np.array_equal(o.cpu().numpy().transpose(0, 2, 1), G)
        Go, _ = shifted_cocg_columns(probs[1], tol=1e-13)
        assert relf(sep[1], Go) <= 1e-9
        # a handle may appear in one job only
        with pytest.raises(rs.RsfdError):
            rs.rsfd_shifted_cocg_regions([jobs[0], jobs[0]])
    finally:
        for h in handles:
            h.close()


def test_full_boundary_and_uneven_regions_full_size_first_iterations(rs):
    """The full-boundary workload (48 x 48 x 160, 64 energies, eta 5e-4) and the six uneven regions
    (32 x 32 x 64 ... 72 x 72 x 112, their own energy sets and eta) at full grid size, all seven in one
    rsfd_shifted_cocg_regions call with their autotuned launch options: after 30 iterations the boundary
    rows of x^(i) for two sampled columns per region equal the oracle's (double-float vectors)."""
    from workloads import make_problem
    probs = [make_problem("full_boundary")] + list(make_problem("uneven_regions"))
    handles, outs, jobs, cols = [], [], [], []
    try:
        for p in probs:
            h = rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=rs.RSFD_DF64)
            c = p.cols[[0, len(p.cols) // 2 + 3]]
            rs.rsfd_autotune(h.ptr, p.energies, p.eta, slots=int(c.size), iters=64)
            o = torch.zeros((p.K, c.size, h.nb), dtype=torch.complex128, device="cuda")
            handles.append(h)
            outs.append(o)
            cols.append(c)
            jobs.append(dict(h=h.ptr, cols=c, energies=p.energies, eta=p.eta, tol=p.tol, maxit=30, G0_bb=o))
        st, per = rs.rsfd_shifted_cocg_regions(jobs)
        torch.cuda.synchronize()
        assert st == rs.RSFD_ERR_NOT_CONVERGED
        for (s, info, _), p, c, o in zip(per, probs, cols, outs):
            assert s == rs.RSFD_ERR_NOT_CONVERGED and (info["iters"] == 30).all()
            Go, res = shifted_cocg_columns(p, cols=c, maxit=30)
            G = o.cpu().numpy().transpose(0, 2, 1)
            assert relf(G, Go) <= 1e-6, p.name
    finally:
        for h in handles:
            h.close()


def test_regions_report_a_failing_region(rs):
    """A region whose arguments are invalid (tol outside (0, 1)) fails alone: its status is the error,
    the other region still solves, and the call returns the error with the region named."""
    p = small_problem(grid=(10, 9, 12), h=0.5, fd_order=2, n_wells=2, n_energies=3, e_range=(0.4, 1.6),
                      eta=5e-2, tol=1e-10, cols=2, seed=8)
    handles = [rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=rs.RSFD_FP64) for _ in range(2)]
    try:
        outs = [torch.zeros((p.K, p.cols.size, h.nb), dtype=torch.complex128, device="cuda") for h in handles]
        jobs = [dict(h=handles[0].ptr, cols=p.cols, energies=p.energies, eta=p.eta, tol=p.tol, maxit=p.maxit,
                     G0_bb=outs[0]),
                dict(h=handles[1].ptr, cols=p.cols, energies=p.energies, eta=p.eta, tol=2.0, maxit=p.maxit,
                     G0_bb=outs[1])]
        with pytest.raises(rs.RsfdError) as e:
            rs.rsfd_shifted_cocg_regions(jobs)
        assert e.value.status == rs.RSFD_ERR_ARG
        assert "region 1" in rs.rsfd_last_error(None)
        torch.cuda.synchronize()
        Go, _ = shifted_cocg_columns(p, tol=1e-12)
        G = outs[0].cpu().numpy().transpose(0, 2, 1)
        assert relf(G, Go) <= 1e-9
    finally:
        for h in handles:
            h.close()


def test_sweep_rejects_an_unwritable_directory(rs, tmp_path):
    p = small_problem(grid=(8, 7, 10), h=0.5, fd_order=2, n_wells=1, n_energies=2, eta=5e-2, tol=1e-8, cols=2)
    with rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=rs.RSFD_FP64) as h:
        G = torch.zeros((p.K, p.cols.size, h.nb), dtype=torch.complex128, device="cuda")
        with pytest.raises(rs.RsfdError) as e:
            rs.rsfd_shifted_cocg_sweep(h.ptr, p.cols, p.energies, p.eta, p.tol, p.maxit, G, 1,
                                       str(tmp_path / "missing" / "dir"))
        assert e.value.status == rs.RSFD_ERR_ARG
