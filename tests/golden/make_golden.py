"""Write the stored expected values of the full-size parity tests by running the CPU oracle.

This script calls only ``oracle/`` (and the seeded inputs of ``workloads``); nothing it stores
comes from the CUDA library.  Output, for the 64x64x128 "sampled_columns_mixed" workload:

* ``sampled_columns_mixed_golden.npz``: for the first ``--ncols`` columns of the workload, the
  oracle's G0_bb (tol 1e-10, FP64) on every 64th boundary row and every energy, and the same at the
  workload's own tolerance (``G0_loose``).
* ``sampled_columns_mixed_oracle_iterations.json``: the oracle's seed iterations per column at the
  workload's own tolerance (used to scale the bounded CPU-baseline sample in bench.py).

For the 8x8x12 "tiny_wire_fp64" workload (``--workload tiny_wire_fp64``, seconds):

* ``tiny_wire_fp64_golden.npz``: the oracle's dense G_bb = [(Z - H_T - Sigma_L - Sigma_R)^{-1}]_{bb}
  (Eq. GF2, LU) for every energy, with the lead self-energies of the oracle's closed form, and the
  Fisher-Lee T(E) (Eq. TF) computed from it.

Run:  python tests/golden/make_golden.py --ncols 2   (about an hour of single-core CPU time)
      python tests/golden/make_golden.py --workload tiny_wire_fp64
"""

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from workloads import make_problem                     # noqa: E402
from oracle.cocg import shifted_cocg                   # noqa: E402
from oracle.operator import hamiltonian, apply_h, boundary_rows   # noqa: E402


def one_column(args):
    name, j, tol, row_stride = args
    p = make_problem(name)
    H, P, wE = hamiltonian(p)
    rows = boundary_rows(p.grid, p.n_face)[::row_stride]
    b = np.zeros(p.N, np.complex128)
    b[j] = 1.0
    t0 = time.time()
    r = shifted_cocg(lambda v: apply_h(H, P, wE, v), b, p.energies + 1j * p.eta, tol, rows=rows, maxit=400000)
    return j, r.x, r.iterations, r.switches, r.status, time.time() - t0


def tiny_wire(name):
    from oracle.dense import g_dense
    from oracle.leads import sigma_bloch
    from oracle.transmission import transmission
    p = make_problem(name)
    b = boundary_rows(p.grid, p.n_face)
    G, T = [], []
    for E in p.energies:
        Z = E + 1j * p.eta
        SL, SR = sigma_bloch(p.grid[0], p.grid[1], p.h, p.fd_order, Z)
        Gd = g_dense(p, Z, SL, SR, rows=b, cols=b)
        G.append(Gd)
        T.append(transmission(Gd, SL, SR)[0])
    np.savez_compressed(os.path.join(HERE, f"{name}_golden.npz"), rows=b, energies=p.energies, eta=p.eta,
                        G_bb=np.stack(G), T=np.array(T))
    print("done", name, np.array(T))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="sampled_columns_mixed")
    ap.add_argument("--ncols", type=int, default=2)
    ap.add_argument("--row-stride", type=int, default=64)
    ap.add_argument("--procs", type=int, default=4)
    args = ap.parse_args()
    if args.workload == "tiny_wire_fp64":
        tiny_wire(args.workload)
        return
    p = make_problem(args.workload)
    cols = [int(c) for c in p.cols[:args.ncols]]
    jobs = [(args.workload, j, 1e-10, args.row_stride) for j in cols]
    jobs += [(args.workload, j, p.tol, args.row_stride) for j in cols]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(args.procs, len(jobs))) as pool:
        out = pool.map(one_column, jobs)
    tight = out[:len(cols)]
    loose = out[len(cols):]
    rows = boundary_rows(p.grid, p.n_face)[::args.row_stride]
    np.savez_compressed(os.path.join(HERE, f"{args.workload}_golden.npz"),
                        cols=np.array(cols), rows=rows, row_stride=args.row_stride,
                        G0=np.stack([o[1] for o in tight], axis=-1),        # [K, nrows, ncols]
                        iterations=np.array([o[2] for o in tight]), tol=1e-10,
                        G0_loose=np.stack([o[1] for o in loose], axis=-1),  # the oracle at the workload's tol
                        tol_loose=p.tol)
    json.dump({"workload": args.workload, "tol": p.tol, "columns": cols,
               "iterations": [int(o[2]) for o in loose], "switches": [int(o[3]) for o in loose],
               "status": [int(o[4]) for o in loose], "seconds": [round(o[5], 1) for o in loose],
               "mean_iterations": float(np.mean([o[2] for o in loose])),
               "note": "seed iterations of the FP64 CPU oracle per column at the workload tolerance"},
              open(os.path.join(HERE, f"{args.workload}_oracle_iterations.json"), "w"), indent=1)
    print("done", [(o[0], o[2], o[4], round(o[5])) for o in out])


if __name__ == "__main__":
    main()
