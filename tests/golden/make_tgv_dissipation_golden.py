"""Write tests/golden/tgv8_k5_dissipation.json: the FP64 oracle's kinetic-energy history of the
Taylor--Green vortex (Sec. 4.2) on 8^3 cells, k = 5 (nq_conv 8, nq_visc 6), Re = 1600, Ma = 0.1,
integrated with RK(5,4) to t = 2.

Calls only the oracle (and the seeded input module for the closed-form initial field).  The time
step restates Eq. TimeStepRestrictions_Compressible: dt = min(Cr / k^1.5 h / (U0 + c), D / k^3 h^2 / nu)
with Cr = 0.4, D = 0.02, h = 2 pi / 8 (the cells' edge), c = U0 / Ma, nu = U0 L / Re.  Every `every`
steps the sample (e_k, eps, -de_k/dt) is taken from the oracle's diagnostics with L(U) of that state,
which is also the first stage's evaluation of the next step.

    python tests/golden/make_tgv_dissipation_golden.py     (about an hour of CPU)
"""
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import diagnostics as odiag  # noqa: E402
from oracle import physics as ph  # noqa: E402
from oracle import rk as ork  # noqa: E402
from oracle.mesh import BoxMesh  # noqa: E402
from oracle.operator import DGOperator  # noqa: E402
from paper_1806_03095_gb300 import inputs  # noqa: E402

K, NCELL, T_FINAL, EVERY = 5, 8, 2.0, 8
RE, MA, CR, D = 1600.0, 0.1, 0.4, 0.02


def main(out=os.path.join(HERE, "tgv8_k5_dissipation.json")):
    lo, hi = (-math.pi,) * 3, (math.pi,) * 3
    op = DGOperator(BoxMesh((NCELL,) * 3, lo, hi, (1, 1, 1), K), ph.Physics.from_numbers(RE, 0.71, MA),
                    (3 * K) // 2 + 1, K + 1)
    h, u0 = 2.0 * math.pi / NCELL, 1.0
    dt = min(CR / K ** 1.5 * h / (u0 + u0 / MA), D / K ** 3 * h * h / (u0 * 1.0 / RE))
    nsteps = int(round(T_FINAL / dt))
    U = inputs.tgv_state(op.xyz)
    dU = U * 0.0
    samples = []
    t0 = time.time()
    for n in range(nsteps + 1):
        LU = op.L(U)
        if n % EVERY == 0:
            d = odiag.diagnostics(op, U, LU)
            samples.append([n, n * dt, float(d[0]), float(d[1]), float(d[2])])
            print("step %d/%d  -dek/dt %.12e  (%.0f s)" % (n, nsteps, float(d[2]), time.time() - t0), flush=True)
        if n == nsteps:
            break
        for i in range(ork.STAGES):
            L = LU if i == 0 else op.L(U)
            dU = ork.A[i] * dU + dt * L
            U = U + ork.B[i] * dU
    with open(out, "w") as f:
        json.dump({"quantity": "oracle e_k, eps, -de_k/dt of TGV %d^3, k = %d, RK(5,4) to t = %g" % (NCELL, K, T_FINAL),
                   "written_by": "tests/golden/make_tgv_dissipation_golden.py (oracle only)",
                   "dt": dt, "every": EVERY, "nsteps": nsteps,
                   "columns": ["step", "t", "e_k", "eps", "-de_k/dt"], "samples": samples}, f, indent=0)


if __name__ == "__main__":
    main()
