"""GPU parity of the tensor-core form of the Dyson step (Eq. sec3-01a restricted to the boundary rows):
the 3xTF32 batched complex GEMM (tcgen05) against an FP64 matrix product of the same FP32 inputs, and
the FP32 LU / triangular solves with FP64 refinement against the oracle's dense Dyson solve."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from workloads import random_complex_matrices   # noqa: E402
from oracle.dyson import dyson_solve             # noqa: E402
from oracle.transmission import transmission     # noqa: E402


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_00081_gb300.build_lib import build
    build()
    import paper_1502_00081_gb300 as m
    m.load_library()
    return m


def _rand_c64(shape, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)).astype(np.complex64)


def _abi(M):
    """[K, rows, cols] matrices -> contiguous column-major ABI layout on the GPU."""
    return torch.from_numpy(np.ascontiguousarray(M.transpose(0, 2, 1))).cuda()


def _mat(t):
    return t.cpu().numpy().astype(np.complex128).transpose(0, 2, 1)


# (m, n, k): single tile, ragged in every dimension, several tiles in m and n, K not a multiple of 16
GEMM_SHAPES = [(1, 1, 1), (16, 16, 8), (70, 33, 17), (128, 128, 64), (200, 300, 100), (257, 129, 65)]


@pytest.mark.parametrize("m,n,k", GEMM_SHAPES)
@pytest.mark.parametrize("beta", [0.0, 1.0])
def test_cgemm_tf32x3_matches_fp64_product(rs, m, n, k, beta):
    """C = alpha A B + beta C in 3xTF32 equals the FP64 product of the FP32 inputs to FP32-class accuracy
    (a single TF32 product would be ~1e-3 off: the bound pins the hi/lo split)."""
    batch, alpha = 3, 0.75 - 0.5j
    A = _rand_c64((batch, m, k), 1)
    B = _rand_c64((batch, k, n), 2)
    C = _rand_c64((batch, m, n), 3)
    At, Bt, Ct = _abi(A), _abi(B), _abi(C)
    rs.rsfd_cgemm_tf32x3(At, Bt, Ct, alpha=alpha, beta=beta)
    torch.cuda.synchronize()
    got = _mat(Ct)
    ref = alpha * np.einsum("bik,bkj->bij", A.astype(np.complex128), B.astype(np.complex128))
    if beta:
        ref = ref + C.astype(np.complex128)
    for b in range(batch):
        err = np.linalg.norm(got[b] - ref[b]) / np.linalg.norm(ref[b])
        assert err <= 2e-6, (b, err)


def test_cgemm_tf32x3_argument_errors(rs):
    lib = rs.load_library()
    import ctypes
    al = (ctypes.c_double * 2)(1.0, 0.0)
    # k = 0, beta not in {0, 1}, leading dimension too small: rejected before any launch
    assert lib.rsfd_cgemm_tf32x3(1, 4, 4, 0, al, 1, 4, 16, 1, 4, 16, 0.0, 1, 4, 16, None) == rs.RSFD_ERR_ARG
    assert lib.rsfd_cgemm_tf32x3(1, 4, 4, 4, al, 1, 4, 16, 1, 4, 16, 0.5, 1, 4, 16, None) == rs.RSFD_ERR_ARG
    assert lib.rsfd_cgemm_tf32x3(1, 4, 4, 4, al, 1, 3, 16, 1, 4, 16, 0.0, 1, 4, 16, None) == rs.RSFD_ERR_ARG


def _dyson_gpu(rs, G0, SL, SR, kind, refine=0):
    K, nb = G0.shape[0], G0.shape[1]
    ns = nb // 2
    with rs.Handle((ns, 1, 4), 0.5, 2, np.zeros(ns * 4), n_face=1, precision=rs.RSFD_FP64) as h:
        assert h.nb == nb
        rs.rsfd_set_solve_options(h.ptr, dyson_kind=kind, dyson_refine=refine)
        G = torch.empty((K, nb, nb), dtype=torch.complex128, device="cuda")
        ref = rs.rsfd_dyson_boundary(h.ptr, _abi(G0), _abi(SL), _abi(SR), G)
        T = rs.rsfd_transmission(h.ptr, G, _abi(SL), _abi(SR))
        return _mat(G), ref, T


@pytest.mark.parametrize("nb", [16, 70, 128, 200, 520])
def test_dyson_tensor_core_matches_oracle(rs, nb):
    """FP32 LU on the tensor cores + two FP64 refinement steps reaches the FP64 oracle's Dyson solve
    (several LU panels and GEMM tiles with ragged edges at nb = 200, 520)."""
    K, ns = 3, nb // 2
    G0 = random_complex_matrices(nb, K, seed=21, scale=0.5)
    SL = random_complex_matrices(ns, K, seed=22, scale=0.5, imag_sign=-1)
    SR = random_complex_matrices(ns, K, seed=23, scale=0.5, imag_sign=-1)
    Gg, ref, T = _dyson_gpu(rs, G0, SL, SR, rs.RSFD_DYSON_TC)
    for k in range(K):
        Go = dyson_solve(G0[k], SL[k], SR[k])
        assert np.linalg.norm(Gg[k] - Go) / np.linalg.norm(Go) <= 1e-10
        assert abs(T[k] - transmission(Go, SL[k], SR[k])[0]) <= 1e-9 * max(1.0, abs(T[k]))
    assert (ref < 1e-12).all(), ref


def test_dyson_tensor_core_one_refinement_step(rs):
    """One FP64 refinement step already brings the FP32 tensor-core solve well below the mixed-mode
    tolerance (1e-5 on G_bb)."""
    nb, K = 256, 2
    G0 = random_complex_matrices(nb, K, seed=31, scale=0.5)
    SL = random_complex_matrices(nb // 2, K, seed=32, scale=0.5, imag_sign=-1)
    SR = random_complex_matrices(nb // 2, K, seed=33, scale=0.5, imag_sign=-1)
    Gg, ref, _ = _dyson_gpu(rs, G0, SL, SR, rs.RSFD_DYSON_TC, refine=1)
    for k in range(K):
        Go = dyson_solve(G0[k], SL[k], SR[k])
        assert np.linalg.norm(Gg[k] - Go) / np.linalg.norm(Go) <= 1e-7
    assert (ref < 1e-8).all(), ref
