"""Run by test_gpu_debug.py in a process of its own with CGH_LIB_VARIANT=debug: the small parity cases through
the debug build of the library (device-side bounds checks latch CGH_EBOUNDS instead of faulting).  Every call
must return CGH_OK and every hologram must meet its tolerance against the oracle."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from paper_1309_2734_gb300 import Hologram, _lib, batch, workloads  # noqa: E402

NRMS = {"direct_sfu": 1e-5, "direct_accurate": 1e-5, "gemm_f16": 2e-3, "gemm_bf16": 1e-2, "gemm_split16": 1e-5}


def main():
    assert os.path.basename(_lib.LIB_PATH) == "libcgh_debug.so", _lib.LIB_PATH
    torch.cuda.set_device(0)
    cases = [workloads.small_direct()] + [workloads.random_cloud(1000 + w + n, w, h, n)
                                          for w, h, n in [(257, 33, 300), (31, 300, 256), (1000, 3, 77)]]
    for c in cases:
        ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, c.width, c.height)
        xyz, amp = torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda()
        for form, tol in NRMS.items():
            with Hologram(c.width, c.height, c.pitch_m, c.lambda_m, form=form) as h:
                f = h.point_cloud(xyz, amp)
                h.sync()   # raises on CGH_EBOUNDS
            err = oracle.nrms(f.cpu().numpy(), ref)
            assert err <= tol, (c.name, form, err)
    # a persistent batch mixing every form's units (direct chunks folded, GEMM K chunks ordered)
    clouds = [workloads.random_cloud(720, 300, 200, 5000), workloads.random_cloud(722, 130, 257, 9000),
              workloads.random_cloud(723, 64, 64, 0)]
    dev = [(torch.from_numpy(c.xyz).cuda(), torch.from_numpy(c.amp).cuda(), c.width, c.height, c.pitch_m,
            c.lambda_m) for c in clouds]
    for form in ("direct_sfu", "gemm_split16"):
        outs = [torch.zeros((c.height, c.width), device="cuda") for c in clouds]
        with Hologram(8, 8, 8e-6, 532e-9, form=form) as h:
            h.set_option(_lib.CGH_OPT_GEMM_CHUNK, 2)
            batch(h, dev, outs)
            h.sync()
        for c, o in zip(clouds, outs):
            if c.n_points:
                ref = oracle.field(c.pitch_m, c.lambda_m, c.xyz, c.amp, c.width, c.height)
                assert oracle.nrms(o.cpu().numpy(), ref) <= NRMS[form], (c.name, form)
            else:
                assert torch.count_nonzero(o).item() == 0
    print("debug build: all cases clear")


if __name__ == "__main__":
    main()
