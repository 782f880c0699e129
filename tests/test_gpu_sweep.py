"""GPU checks of the checkpointed column sweep (rsfd_shifted_cocg_sweep) around the shifted COCG of
Sec. III B: the blocks' results equal a direct solve and the oracle; a rerun resumes from the block
files, recomputing only the missing block; changed inputs invalidate the files."""

import os

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


def test_sweep_checkpoints_and_resumes(rs, tmp_path):
    p = small_problem(grid=(14, 11, 16), h=0.5, fd_order=4, n_wells=3, n_energies=5, e_range=(0.4, 2.0),
                      eta=5e-2, tol=1e-12, cols=7)
    d = str(tmp_path)
    with rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=rs.RSFD_FP64) as h:
        G = torch.zeros((p.K, p.cols.size, h.nb), dtype=torch.complex128, device="cuda")
        st, info, resumed = rs.rsfd_shifted_cocg_sweep(h.ptr, p.cols, p.energies, p.eta, p.tol, p.maxit, G, 3, d)
        assert st == rs.RSFD_OK and resumed == 0
        assert sorted(os.listdir(d)) == ["g0_block_000000.bin", "g0_block_000001.bin", "g0_block_000002.bin"]
        G1 = G.cpu().numpy().copy()
        # the same columns solved directly
        Gd = torch.zeros_like(G)
        st2, info2, _ = rs.rsfd_shifted_cocg(h.ptr, p.cols, p.energies, p.eta, p.tol, p.maxit, Gd)
        assert st2 == rs.RSFD_OK
        assert np.abs(G1 - Gd.cpu().numpy()).max() <= 1e-12 * np.abs(G1).max()
        assert np.array_equal(info["iters"], info2["iters"])
        # rerun: every block comes from its file, bit for bit
        G.zero_()
        st, info3, resumed = rs.rsfd_shifted_cocg_sweep(h.ptr, p.cols, p.energies, p.eta, p.tol, p.maxit, G, 3, d)
        assert resumed == 3 and np.array_equal(G.cpu().numpy(), G1) and np.array_equal(info3, info)
        # a lost block is recomputed, the others are read back
        os.remove(os.path.join(d, "g0_block_000001.bin"))
        G.zero_()
        st, info4, resumed = rs.rsfd_shifted_cocg_sweep(h.ptr, p.cols, p.energies, p.eta, p.tol, p.maxit, G, 3, d)
        assert resumed == 2 and np.array_equal(G.cpu().numpy(), G1)
        # other inputs (a different tolerance) do not reuse the files
        st, info5, resumed = rs.rsfd_shifted_cocg_sweep(h.ptr, p.cols, p.energies, p.eta, 1e-10, p.maxit, G, 3, d)
        assert resumed == 0
    Go, _ = shifted_cocg_columns(p, tol=1e-13)
    assert np.linalg.norm(G1.transpose(0, 2, 1) - Go) / np.linalg.norm(Go) <= 1e-9


def test_sweep_to_files_then_energy_chunks_through_dyson(rs, tmp_path):
    """A sweep that keeps G0_bb only in its block files (no device G0_bb), then energy chunks read back
    across all column blocks: each chunk equals the in-memory solve's energies, and the Dyson step on a
    chunk gives the same G_bb and T as on the whole G0_bb."""
    p = small_problem(grid=(8, 7, 12), h=0.5, fd_order=2, n_wells=2, n_energies=5, e_range=(0.5, 2.0),
                      eta=4e-2, tol=1e-12)
    d = str(tmp_path)
    with rs.Handle(p.grid, p.h, p.fd_order, p.V, n_face=p.n_face, precision=rs.RSFD_FP64) as h:
        cols = h.rows
        st, info, resumed = rs.rsfd_shifted_cocg_sweep(h.ptr, cols, p.energies, p.eta, p.tol, p.maxit, None, 40, d)
        assert st == rs.RSFD_OK and resumed == 0 and len(os.listdir(d)) == 3
        Gfull = torch.zeros((p.K, cols.size, h.nb), dtype=torch.complex128, device="cuda")
        rs.rsfd_shifted_cocg(h.ptr, cols, p.energies, p.eta, p.tol, p.maxit, Gfull)
        part = torch.zeros((2, cols.size, h.nb), dtype=torch.complex128, device="cuda")
        rs.rsfd_sweep_load_energies(h.ptr, cols, p.energies, p.eta, p.tol, p.maxit, 40, d, 2, 2, part)
        torch.cuda.synchronize()
        assert (torch.abs(part - Gfull[2:4]).max() <= 1e-12 * torch.abs(Gfull).max()).item()
        SLh, SRh = rs.rsfd_lead_sigma_uniform(p.grid[0], p.grid[1], p.h, p.fd_order, p.energies, p.eta)
        SL, SR = torch.from_numpy(SLh).cuda(), torch.from_numpy(SRh).cuda()
        G = torch.empty_like(Gfull)
        rs.rsfd_dyson_boundary(h.ptr, Gfull, SL, SR, G)
        T = rs.rsfd_transmission(h.ptr, G, SL, SR)
        Gp = torch.empty_like(part)
        rs.rsfd_dyson_boundary(h.ptr, part, SL[2:4].contiguous(), SR[2:4].contiguous(), Gp)
        Tp = rs.rsfd_transmission(h.ptr, Gp, SL[2:4].contiguous(), SR[2:4].contiguous())
        assert np.abs(Tp - T[2:4]).max() <= 1e-10
        # other inputs: the files do not match
        with pytest.raises(rs.RsfdError):
            rs.rsfd_sweep_load_energies(h.ptr, cols, p.energies, p.eta, 1e-9, p.maxit, 40, d, 0, 1, part)
