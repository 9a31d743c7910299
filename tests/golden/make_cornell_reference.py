"""Write the high-sample reference image of the Cornell-box configuration
(64 x 64, depth 8) used to measure RMSE of GPU renders: the FP64 oracle at
2^15 samples per pixel, seed 0, Gaussian filter sigma 0.5. Calls only
oracle/ and the input generator.

    python tests/golden/make_cornell_reference.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1705_01263_gb300 import scenes  # noqa: E402

SPP = 1 << 15


def main():
    sd, cam = scenes.cornell_box()
    s = oracle.Scene(sd)
    t0 = time.time()
    S, S2, C, rays = s.render(cam, SPP, 8)
    mean, var = oracle.resolve(S, S2, C)
    np.savez_compressed(os.path.join(HERE, "cornell_64_depth8_ref.npz"), mean=mean, var=var, spp=SPP,
                        seconds=time.time() - t0)
    print(f"{SPP} spp in {time.time() - t0:.1f} s, mean {mean.mean(axis=(0, 1))}")


if __name__ == "__main__":
    main()
