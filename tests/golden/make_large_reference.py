"""Writes the exact-exponential reference values of the large transmon-cavity workloads.

Every value comes from ``oracle/`` alone (nothing from the CUDA path):

* ``c3_gate_d4000_n3_dense.txt``   two transmons (4 levels) x cavity (250 levels), d = 4000, first
  3 steps of the seeded controls: ``oracle.cost_and_grad`` (dense ``eigh`` propagators and the
  divided-difference derivative of App. F).
* ``c3_gate_d4000_full_exact.txt`` the same workload at its full N = 2000:
  ``oracle.sparse_reference.cost_and_grad`` (exponential actions by ``expm_multiply``, derivative
  by the auxiliary block matrix of Sec. III.B).  At N = 3 the script checks it against the dense
  oracle above before writing anything.
* ``c4_gate_d16000_n3_exact.txt``  two transmons x cavity (1000 levels), d = 16,000, 16 states,
  first 3 steps: ``oracle.sparse_reference.cost_and_grad``.
* ``dense_gue_q11_n2_dense.txt``   11-qubit register with a dense GUE drift (every H_ij non-zero),
  d = 2048, 16 states, first 2 steps: ``oracle.cost_and_grad``.

Each file: comment lines, then ``cost``, ``C1``, ``C2``, ``C_amp``, then the K x N gradient, one
row per control.  Run:  python tests/golden/make_large_reference.py [--workers 8]
"""

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def write(name, problem, res, how):
    path = os.path.join(HERE, name)
    K, N = res.grad.shape
    with open(path, "w") as fh:
        fh.write(f"# {problem.name}: d={problem.dim}, K={K}, n={problem.n_states}, N={N}, dt={problem.dt}, "
                 f"seed={problem.meta.get('seed')}, controls = the workload's seeded u0\n")
        fh.write(f"# {how}\n")
        fh.write("# cost C1 C2 C_amp, then the gradient dC/du_kn, row k = control k (Sec. II composite cost)\n")
        fh.write(f"{res.cost:.17e} {res.parts['C1']:.17e} {res.parts['C2']:.17e} {res.parts['C_amp']:.17e}\n")
        for k in range(K):
            fh.write(" ".join(f"{v:.17e}" for v in res.grad[k]) + "\n")
    print(f"wrote {path}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", default="", help="comma list of: c3n3, c3full, c4n3, dense2")
    args = ap.parse_args()
    only = set(filter(None, args.only.split(",")))
    from oracle import cost_and_grad as dense_cost_and_grad
    from oracle import sparse_reference
    from workloads import build_config, dense_register_gate

    if not only or "c3n3" in only or "c3full" in only:
        p3 = build_config("c3_gate_d4000", n_steps=3)
        t = time.time()
        dense = dense_cost_and_grad(p3, p3.u0)
        print(f"dense oracle, d = 4000, N = 3: {time.time() - t:.0f} s")
        sparse = sparse_reference.cost_and_grad(p3, p3.u0)
        dc = abs(dense.cost - sparse.cost) / abs(dense.cost)
        dg = np.linalg.norm(dense.grad - sparse.grad) / np.linalg.norm(dense.grad)
        print(f"sparse reference vs dense oracle at N = 3: cost {dc:.2e}, gradient {dg:.2e}")
        assert dc < 1e-13 and dg < 1e-12, (dc, dg)
        if not only or "c3n3" in only:
            write("c3_gate_d4000_n3_dense.txt", p3, dense,
                  "oracle.cost_and_grad (dense eigh propagators, App. F divided differences)")
    if not only or "c3full" in only:
        p = build_config("c3_gate_d4000")
        t = time.time()
        res = sparse_reference.cost_and_grad(p, p.u0, workers=args.workers)
        print(f"sparse reference, d = 4000, N = {p.n_steps}: {time.time() - t:.0f} s")
        write("c3_gate_d4000_full_exact.txt", p, res,
              "oracle.sparse_reference.cost_and_grad (expm_multiply actions, auxiliary block-matrix derivative)")
    if not only or "c4n3" in only:
        p4 = build_config("c4_gate_d16000", n_steps=3)
        t = time.time()
        res = sparse_reference.cost_and_grad(p4, p4.u0, workers=args.workers)
        print(f"sparse reference, d = 16000, N = 3: {time.time() - t:.0f} s")
        write("c4_gate_d16000_n3_exact.txt", p4, res,
              "oracle.sparse_reference.cost_and_grad (expm_multiply actions, auxiliary block-matrix derivative)")
    if not only or "dense2" in only:
        pd = dense_register_gate(n_steps=2)
        t = time.time()
        res = dense_cost_and_grad(pd, pd.u0)
        print(f"dense oracle, d = 2048 dense drift, N = 2: {time.time() - t:.0f} s")
        write("dense_gue_q11_n2_dense.txt", pd, res,
              "oracle.cost_and_grad (dense eigh propagators, App. F divided differences)")


if __name__ == "__main__":
    main()
