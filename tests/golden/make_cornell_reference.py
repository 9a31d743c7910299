"""Write the high-sample reference images of the Cornell-box configuration
(64 x 64, depth 8) used to measure RMSE of GPU renders: the FP64 oracle at
2^15 samples per pixel from sequence iteration 2^20 on (so that renders from
iteration 0, on the GPU or not, share no sample with it: a reference drawn
from the same samples would understate their error), seed 0, Gaussian
filter sigma 0.5, for the emitter
under the ceiling facing down (cornell_64_depth8_ref.npz) and facing the
ceiling (cornell_up_64_depth8_ref.npz). Calls only oracle/ and the input
generator.

    python tests/golden/make_cornell_reference.py [down|up]
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
ITER0 = 1 << 20


def main(lights):
    for light in lights:
        sd, cam = scenes.cornell_box(light=light)
        s = oracle.Scene(sd)
        t0 = time.time()
        S, S2, C, rays = s.render(cam, SPP, 8, iter0=ITER0)
        mean, var = oracle.resolve(S, S2, C)
        name = "cornell_64_depth8_ref.npz" if light == "down" else "cornell_up_64_depth8_ref.npz"
        np.savez_compressed(os.path.join(HERE, name), mean=mean, var=var, spp=SPP, iter0=ITER0,
                            seconds=time.time() - t0)
        print(f"{light}: {SPP} spp in {time.time() - t0:.1f} s, mean {mean.mean(axis=(0, 1))}")


if __name__ == "__main__":
    main(sys.argv[1:] or ["down", "up"])
