"""Write oracle_iterations.json: FGMRES steps the FP64 oracle needs for one forward and one
adjoint solve of angle 0 of a workload, at the contrast the bench step is evaluated at
(0.9 x the ground-truth phantom).  Calls only the oracle and the input generators.

    python tests/golden/make_oracle_iterations.py ellipses576
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iterations.json")


def main(name):
    w = W.WORKLOADS[name]
    p = O.Problem.from_workload(w)
    f_gt = W.phantom(w)
    th = float(W.angles(w)[0])
    rec = W.receivers(w, f_gt)
    kw = dict(levels=w.levels, nu1=w.nu1, nu2=w.nu2, omega=w.omega, shift=complex(w.shift_re, w.shift_im),
              restart=w.restart, tol=w.tol, maxit=20000)
    gt = O.MGHSolver(p, f_gt, **kw)
    u_gt, _ = gt.solve(O.rhs(p, f_gt, th))
    y = O.sample(u_gt, rec)
    s = O.MGHSolver(p, 0.9 * f_gt, **kw)
    u, info_f = s.solve(O.rhs(p, 0.9 * f_gt, th))
    r, _ = O.misfit(O.sample(u, rec), y)
    G = np.zeros(p.ny * p.nx, dtype=np.complex128)
    G[rec] = np.conj(r)
    _, info_a = s.solve(G.reshape(p.ny, p.nx))
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data[name] = {"angle_index": 0, "contrast": "0.9 x ground-truth phantom", "tol": w.tol, "restart": w.restart,
                  "levels": w.levels, "nu": [w.nu1, w.nu2],
                  "forward_iterations": info_f.iterations, "adjoint_iterations": info_a.iterations,
                  "forward_converged": info_f.converged, "adjoint_converged": info_a.converged}
    with open(OUT, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    print(name, data[name])


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "ellipses576")
