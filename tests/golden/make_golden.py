"""Write the stored expected values used by the GPU parity tests.

Calls only the FP64 oracle (oracle/) on seeded inputs from the shared generators;
nothing here touches the CUDA path.

c1_progot.npz: the 2-D Gaussian workload (n = m = 512, x ~ N(0, I), y = A z + b,
A = [[2, .5], [.5, 1]], b = (1, -1), seed 0), K = 4 constant-speed steps, eps_k from
the oracle's Alg. 4 (held-out target draw, s_p = 2^-3..2^3, beta0 = 5), tau = 1e-6.
Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import progot_oracle as O  # noqa: E402
from paper_2406_05061_gb300 import workloads as W  # noqa: E402


def c1():
    p = W.gaussian_affine(512, 512, 0)
    K = 4
    tau = 1e-6
    al = O.alpha_schedule(K)
    yt = W.heldout_target(p)
    eps, info = O.eps_schedule(p.x, None, p.y, yt, al, tau=tau)
    r = O.progot(None, p.x, None, p.y, eps, al, [tau] * K)
    np.savez(os.path.join(HERE, "c1_progot.npz"), eps=eps, alpha=al, tau=np.full(K, tau), x_out=r.x_out,
             x_last=r.x_last, g_all=r.g_all, f_last=r.f_last, iters=np.array(r.iters), errs=np.array(r.errs),
             eps0=info["eps0"], sigma=info["sigma"], scores=np.array(info["errors"]), p_star=info["p_star"],
             x_steps=np.stack(r.x_steps))


if __name__ == "__main__":
    c1()
    print("wrote", os.path.join(HERE, "c1_progot.npz"))
