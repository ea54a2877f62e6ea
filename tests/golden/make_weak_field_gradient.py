"""Writes weak_field_gradient.txt: the oracle's loss and its exact directional derivatives for the ten-step
density-matching loss on the 64^3 weak-field block (the adjoint benchmark's gradient).

J = 1/2 sum over interior cells of (D~_10 - T)^2, where D~_10 is the conserved density after ten classical RK4
steps (Sec. 3.12) from the initial data (rho, p, v^i | A_i, Psi) of the seeded workload, and T the seeded target.
For each seeded direction d in the initial data (rho, v^i, A_i; the pressure is held fixed), dJ/dd =
sum (D~_10 - T) dD~_10 with dD~_10 carried by the oracle's forward-mode dual numbers through prim->cons and the
ten steps (the recovery differentiated at its root).  This is the derivative of the branch every limiter is on,
which is what the adjoint computes; it has no finite-difference error.

Runs only the oracle (about 4 minutes per direction on 8 threads): python tests/golden/make_weak_field_gradient.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2406_11669_gb300 import workloads as W  # noqa: E402

NSTEPS = 10


def main():
    O.set_threads(int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1)))
    w = W.weak_field_modes()
    M = O.metric_array(w)
    T = W.weak_field_target(w)
    g, n = w.g, w.n
    inter = (slice(g, g + n[2]), slice(g, g + n[1]), slice(g, g + n[0]))
    lines = []
    for name, dP, dA in W.gradient_directions(w):
        # ghost fill (the direction too: periodic images carry the perturbation of the entry they copy), then
        # prim->cons and its derivative
        U, P = O.initial_state(w)
        U[:5] = 0.0
        O.ghost_fill_state(w, U)
        dU = np.zeros_like(U)
        dU[5:8] = dA
        O.ghost_fill_state(w, dU)
        dU[:5] = O.prim2con_jvp(w, M, U, dU[5:8], P, dP)
        Pw = P.copy()
        for _ in range(NSTEPS):
            U, dU = O.rk4_jvp(w, M, U, dU, Pw)
        r = U[0][inter] - T[inter]
        J = 0.5 * float(np.sum(r * r))
        dJ = float(np.sum(r * dU[0][inter]))
        lines.append(f"{name} {J!r} {dJ!r}")
        print(lines[-1], flush=True)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weak_field_gradient.txt")
    with open(out, "w") as f:
        f.write("# weak_field_modes 64^3, 10 RK4 steps, J = 1/2 sum_interior (D~_10 - T)^2; written by "
                "make_weak_field_gradient.py (oracle only)\n")
        f.write("# direction J dJ/dd\n")
        for line in lines:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
