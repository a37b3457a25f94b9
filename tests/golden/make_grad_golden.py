"""Write the oracle's gradient of the held-out loss for the 8+2-frame 160x120 workload.

Calls only oracle/ and synth/: the table starts 30% off the generating one
(every sigma and the outlier weight times 1.3); training and held-out rays are
traversed with it; the FP64 oracle gives the loss, its adjoint gradient and
central differences (h = 1e-6) over all n_bins + 1 table entries.  Writes
grad_diff_8x160x120.json beside this script.
Run from the repository root:  python tests/golden/make_grad_golden.py
"""
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import oracle  # noqa: E402
from synth import make_workload  # noqa: E402
from synth.scenes import theta_off  # noqa: E402

H = 1e-6


def main():
    w = make_workload("diff_8x160x120")
    th = theta_off(w.lut)
    tr = oracle.trace_frames(w.grid, w.frames, th)
    ho = oracle.trace_frames(w.grid, w.heldout, th)
    theta = np.r_[th.log_sigma.astype(np.float64), float(th.outlier_w)]
    args = (tr, ho, w.grid.n_voxels, w.prior, w.init_p, w.iters)
    t0 = time.time()
    loss, g_ls, g_w = oracle.grad(th, theta[:-1], theta[-1], *args)

    def f(x):
        return oracle.grad(th, x[:-1], x[-1], *args, with_grad=False)

    fd = [(f(theta + H * e) - f(theta - H * e)) / (2 * H) for e in np.eye(len(theta))]
    out = {"workload": w.name, "table": "generating table with sigma and w times 1.3",
           "edges": int(tr["ray_off"][-1]), "heldout_edges": int(ho["ray_off"][-1]),
           "passes": w.iters, "first_pass_message": w.init_p, "h": H,
           "loss": loss, "grad_adjoint": list(np.r_[g_ls, g_w]), "grad_fd": list(fd),
           "seconds": time.time() - t0}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "grad_diff_8x160x120.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    g, r = np.r_[g_ls, g_w], np.array(fd)
    print(path, "loss", loss, "|adj - fd| / |fd|", np.linalg.norm(g - r) / np.linalg.norm(r))


if __name__ == "__main__":
    main()
