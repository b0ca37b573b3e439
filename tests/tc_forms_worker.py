"""Worker for test_gpu_tc_forms.py: one mixed-precision round trip in a fresh process (the
tensor-core engine form is chosen from CRV_TC_WS when the library first runs a contraction);
saves the curvelet coefficients and the reconstructed map to the given .npz path."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

import paper_1511_05578_gb300 as crv  # noqa: E402
from gpu_util import case, map_from_device, map_to_device  # noqa: E402


def main(out_path, L, spin):
    real = spin == 0
    lam, J0 = 2.0, 1
    _, fmap = case(L, lam, J0, spin, real, seed=21, power=3.0 if spin else 2.0)
    flags = crv.CRV_F_MIXED | crv.CRV_F_W_FP32 | (crv.CRV_F_REAL if real else 0)
    p = crv.Plan(L, lam, J0, spin, flags)
    W, Wphi, out = p.W_tensors(1), p.Wphi_tensor(1), p.map_tensor(1)
    crv.crv_analysis(p.handle, map_to_device(fmap, real), W, Wphi, 1)
    crv.crv_synthesis(p.handle, W, Wphi, out, 1)
    crv.crv_plan_check(p.handle)
    torch.cuda.synchronize()
    arrays = {f"W{j}": W[j].cpu().numpy() for j in range(J0, p.J + 1)}
    arrays["out"] = map_from_device(out, real)
    arrays["map"] = fmap
    np.savez(out_path, **arrays)
    p.close()


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]), int(sys.argv[3]))
