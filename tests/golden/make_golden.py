"""Write the stored expected values used by the GPU parity tests.

Everything here is computed by the CPU oracle (oracle/) from the seeded
workloads (workloads/); nothing comes from the CUDA library.

    python tests/golden/make_golden.py            # writes irka_laplace2d_n10000.json

irka_laplace2d_n10000.json: the 2D-Laplacian IRKA workload (n = 10,000, E = I, SISO,
r = 6, initial shifts logspace(1, 4, 6)), 20 IRKA iterations with the reuse
schedule of Algorithm 4, right-preconditioned BiCGSTAB to 1e-8: the shift
history, BiCGSTAB iteration counts per solve, the final reduced system, and
H_r(i w) on 1000 log-spaced w in [1, 1e5] together with the exact H(i w)
(sparse LU) used as the |H| scale of the 1e-6 criterion.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import irka, operator as op  # noqa: E402

OMEGA = np.logspace(0, 5, 1000)


def c2l(z):
    z = np.asarray(z, dtype=np.complex128).ravel()
    return [[float(v.real), float(v.imag)] for v in z]


def main():
    t0 = time.time()
    wl = W.laplace2d_siso()
    res = irka.irka(wl.A, wl.E, wl.B, wl.C, wl.shifts, iters=wl.irka_iters, mode="reuse", solver="bicgstab",
                    tol=1e-8)
    s = 1j * OMEGA
    Hr = op.transfer_function_reduced(res.Ar, res.Er, res.Br, res.Cr, s)[:, 0, 0]
    H = op.transfer_function(wl.A, wl.E, wl.B, wl.C, s)[:, 0, 0]
    out = {
        "workload": wl.name,
        "iters": wl.irka_iters,
        "omega": "logspace(0, 5, 1000)",
        "shifts_history": [c2l(x) for x in res.shifts_history],
        "bicgstab_iters": res.iters,
        "relres": res.relres,
        "Ar": res.Ar.tolist(), "Er": res.Er.tolist(), "Br": res.Br.tolist(), "Cr": res.Cr.tolist(),
        "Hr": c2l(Hr),
        "H": c2l(H),
        "oracle_seconds": time.time() - t0,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "irka_laplace2d_n10000.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path, "in %.1f s" % (time.time() - t0))


if __name__ == "__main__":
    main()
