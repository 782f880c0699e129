"""The allocation-free Dyson entry point (rsfd_dyson_boundary_noalloc) against the handle-based one.

Callers that cannot allocate device memory (a service whose device memory already belongs to its own
caching allocator, or a plug-in whose host application forbids new allocations) use
rsfd_dyson_boundary_noalloc, whose scratch is a static device array inside the library.  This test calls it through the C ABI twice in a row, with
different inputs, and compares each result with rsfd_dyson_boundary (which allocates its workspace
through its handle) within the tolerance the Dyson tests use.  The second call checks that contents
left in the shared scratch by the first call do not leak into the next result.  The file is named so
that pytest collects it last.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from workloads import random_complex_matrices   # noqa: E402


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_00081_gb300.build_lib import build
    build()
    import paper_1502_00081_gb300 as m
    m.load_library()
    return m


def _abi(M):
    return torch.from_numpy(np.ascontiguousarray(M.transpose(0, 2, 1))).cuda()


@pytest.mark.parametrize("nb,K", [(64, 3), (128, 8)])
def test_noalloc_matches_handle_dyson_twice(rs, nb, K):
    ns = nb // 2
    with rs.Handle((ns, 1, 4), 0.5, 2, np.zeros(ns * 4), n_face=1, precision=rs.RSFD_FP64) as h:
        assert h.nb == nb
        for call, seed in enumerate((21, 37)):
            G0 = _abi(random_complex_matrices(nb, K, seed=seed, scale=0.5))
            SL = _abi(random_complex_matrices(ns, K, seed=seed + 1, scale=0.5, imag_sign=-1))
            SR = _abi(random_complex_matrices(ns, K, seed=seed + 2, scale=0.5, imag_sign=-1))
            G_ref = torch.empty_like(G0)
            ref_res = rs.rsfd_dyson_boundary(h.ptr, G0, SL, SR, G_ref)
            G_na = torch.full_like(G0, complex(float("nan"), 0.0))
            na_res = rs.rsfd_dyson_boundary_noalloc(G0, SL, SR, G_na)
            torch.cuda.synchronize()
            a, b = G_na.cpu().numpy(), G_ref.cpu().numpy()
            assert np.isfinite(a).all()
            err = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert err <= 1e-10, (call, err)
            assert (na_res < 1e-12).all() and (ref_res < 1e-12).all()


def test_noalloc_rejects_oversize(rs):
    nb, K = 1024, 8   # 3*nb*nb*K*16 bytes = 384 MiB > the 32 MiB static scratch
    z = torch.zeros((1,), dtype=torch.complex128, device="cuda")
    with pytest.raises(rs.RsfdError) as e:
        rs.binding.load_library().rsfd_dyson_boundary_noalloc  # symbol present
        import ctypes
        st = rs.binding.load_library().rsfd_dyson_boundary_noalloc(
            nb, K, ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(z.data_ptr()),
            ctypes.c_void_p(z.data_ptr() + 16), None, ctypes.c_void_p(0))
        if st != 0:
            raise rs.RsfdError(st, rs.rsfd_last_error(None))
    assert e.value.status == rs.RSFD_ERR_ARG and "scratch" in str(e.value)
