"""The room lit through a door (scenes.door_room), pinned with the oracle's
ray caster: the room and the side chamber are closed except for the door, so
a segment from inside the room to a point inside the chamber is blocked
exactly when it crosses the dividing wall (x = 1) outside the door opening
(z in [0.55, 0.75], y below 0.65). Light reaches the room only through the
door; this is what makes the scene the case for path guiding."""
import numpy as np

import oracle
from paper_1705_01263_gb300 import scenes

MISS = 0xFFFFFFFF


def test_door_room_is_closed_except_for_the_door():
    sd, _ = scenes.door_room()
    s = oracle.Scene(sd)
    rng = np.random.default_rng(3)
    n = 4000
    # room points between the boxes (x <= ~0.87 after their rotation) and the
    # dividing wall, chamber points away from its walls and its emitter
    a = np.stack([rng.uniform(0.9, 0.99, n), rng.uniform(0.02, 0.98, n), rng.uniform(0.02, 0.98, n)], 1)
    b = np.stack([rng.uniform(1.05, 1.55, n), rng.uniform(0.05, 0.95, n), rng.uniform(0.4, 0.95, n)], 1)
    d = b - a
    length = np.linalg.norm(d, axis=1)
    u = (1.0 - a[:, 0]) / d[:, 0]
    y1, z1 = a[:, 1] + u * d[:, 1], a[:, 2] + u * d[:, 2]
    inside = (y1 > 0.0) & (y1 < 0.65) & (z1 > 0.55) & (z1 < 0.75)
    # leave out segments that graze the door's frame
    clear = (np.minimum.reduce([np.abs(y1 - 0.65), np.abs(z1 - 0.55), np.abs(z1 - 0.75)]) > 1e-3)
    rays = np.concatenate([a, d / length[:, None], np.zeros((n, 1)), (length * (1 - 1e-4))[:, None]], 1)
    prim, _, _, _ = s.trace(rays, any_hit=True)
    blocked = prim != MISS
    assert clear.mean() > 0.95
    assert inside[clear].sum() > 100 and (~inside[clear]).sum() > 100
    assert np.array_equal(blocked[clear], ~inside[clear])


def test_door_room_emitter_is_hidden_from_above_the_door():
    """From room points higher than the door's top, every segment rising to
    the emitter (on the chamber's ceiling, facing down) crosses the dividing
    wall above the opening and is blocked."""
    sd, _ = scenes.door_room()
    s = oracle.Scene(sd)
    rng = np.random.default_rng(4)
    n = 2000
    a = np.stack([rng.uniform(0.05, 0.95, n), rng.uniform(0.66, 0.95, n), rng.uniform(0.05, 0.95, n)], 1)
    e = np.stack([rng.uniform(1.2, 1.4, n), np.full(n, 0.999), rng.uniform(0.5, 0.85, n)], 1)
    d = e - a
    length = np.linalg.norm(d, axis=1)
    rays = np.concatenate([a, d / length[:, None], np.zeros((n, 1)), (length * (1 - 1e-4))[:, None]], 1)
    prim, _, _, _ = s.trace(rays, any_hit=True)
    assert np.all(prim != MISS)
