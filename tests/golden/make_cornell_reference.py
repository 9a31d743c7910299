"""Write the high-sample reference images of the Cornell-box configuration
(64 x 64, depth 8) used to measure RMSE of GPU renders: the FP64 oracle at
2^15 samples per pixel from sequence iteration 2^20 on (so that renders from
iteration 0, on the GPU or not, share no sample with it: a reference drawn
from the same samples would understate their error), seed 0, Gaussian
filter sigma 0.5, for the emitter
under the ceiling facing down (cornell_64_depth8_ref.npz) and facing the
ceiling (cornell_up_64_depth8_ref.npz); and, at 2^17 samples per pixel,
the room lit from a side chamber through a door (cornell_door_64_depth8_ref.npz;
its guided-versus-plain target is the plain tracer at 16,384 spp, so the
reference takes 8 times that). Calls only oracle/ and the input generator.

    python tests/golden/make_cornell_reference.py [down|up|door]
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


SPP_DOOR = 1 << 17
NAMES = {"down": "cornell_64_depth8_ref.npz", "up": "cornell_up_64_depth8_ref.npz",
         "door": "cornell_door_64_depth8_ref.npz"}


def main(lights):
    for light in lights:
        sd, cam = scenes.door_room() if light == "door" else scenes.cornell_box(light=light)
        spp = SPP_DOOR if light == "door" else SPP
        s = oracle.Scene(sd)
        t0 = time.time()
        S, S2, C, rays = s.render(cam, spp, 8, iter0=ITER0)
        mean, var = oracle.resolve(S, S2, C)
        np.savez_compressed(os.path.join(HERE, NAMES[light]), mean=mean, var=var, spp=spp, iter0=ITER0,
                            seconds=time.time() - t0)
        print(f"{light}: {spp} spp in {time.time() - t0:.1f} s, mean {mean.mean(axis=(0, 1))}")


if __name__ == "__main__":
    main(sys.argv[1:] or ["down", "up"])
