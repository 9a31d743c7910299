"""Benchmark of the GB300 QMC path tracer.

Workload (default): the 1,000,000-triangle sphere field (200 noise-displaced
tessellated spheres on a displaced plane, GGX + Lambert layered materials,
256 emissive triangles, 2048 x 1024 procedural sky) rendered at 1920 x 1080,
64 samples per pixel, max depth 16. One step = one full render of that
configuration (132,710,400 camera paths) through rt_render. Inputs are
synthetic and seeded (scenes.sphere_field).

Prints ONE JSON line (rank 0). Multi-GPU (torchrun): every rank renders its
own disjoint iteration range (weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpaths/s"
UNIT = "Mpaths/s"
WORKLOAD = "sphere-field 1M tris, 1920x1080, 64 spp, depth 16"
SPP, DEPTH = 64, 16
# DRAM bytes (read + write) per extension ray of k_trace_ext_simple, measured
# with ncu (dram__bytes_read.sum + dram__bytes_write.sum) over all 17 launches
# of one 4-spp render of the same scene, caches as the program left them:
# 1,967.2 MB for 19,024,373 rays.
TRACE_EXT_DRAM_BYTES_PER_RAY = 105.8


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model():
    """Host CPU model: lscpu's "Model name" (and vendor), else /proc/cpuinfo
    (x86 "model name", Arm implementer / part), else "unknown"."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        kv = dict(l.split(":", 1) for l in out.splitlines() if ":" in l)
        kv = {k.strip(): v.strip() for k, v in kv.items()}
        if kv.get("Model name"):
            return " ".join(x for x in (kv.get("Vendor ID"), kv["Model name"]) if x)
    except (OSError, subprocess.SubprocessError, ValueError):
        pass
    try:
        txt = open("/proc/cpuinfo").read()
    except OSError:
        return "unknown"
    for line in txt.splitlines():
        if line.lower().startswith("model name"):
            return line.split(":", 1)[1].strip()
    impl = [l.split(":", 1)[1].strip() for l in txt.splitlines() if l.startswith("CPU implementer")]
    part = [l.split(":", 1)[1].strip() for l in txt.splitlines() if l.startswith("CPU part")]
    if impl and part:
        return f"Arm implementer {impl[0]} part {part[0]}"
    return "unknown"


def cpu_baseline_oracle(sd, cam):
    """The FP64 oracle as it stands, on all host cores, on a bounded sample of
    the workload: the full scene and image at 8 of the 64 spp (about 10-20 s
    on 16 cores)."""
    import oracle
    t0 = time.time()
    osc = oracle.Scene(sd)
    build_s = time.time() - t0
    from paper_1705_01263_gb300 import scenes as sc_mod
    W, H = 1920, 1080
    spp = 8
    c2 = sc_mod.Camera(cam.eye, cam.look_at, cam.up, cam.vfov_deg, W, H)
    t0 = time.time()
    _, _, cnt, rays = osc.render(c2, spp, DEPTH)
    dt = time.time() - t0
    paths = int(cnt.sum())
    cores = os.cpu_count() or 1
    # one core: the same camera at a quarter of the resolution, 1 spp
    c1 = sc_mod.Camera(cam.eye, cam.look_at, cam.up, cam.vfov_deg, W // 4, H // 4)
    t0 = time.time()
    _, _, cnt1, _ = osc.render(c1, 1, DEPTH, threads=1)
    dt1 = time.time() - t0
    return {"value": paths / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{W}x{H} px x {spp} spp of the same scene and camera (depth {DEPTH}), "
                      f"{paths} paths in {dt:.1f} s; oracle BVH build {build_s:.1f} s not timed",
            "mrays_per_s": rays / dt / 1e6, "cpu": cpu_model(),
            "one_core": {"value": int(cnt1.sum()) / dt1 / 1e6, "unit": UNIT, "cores": 1,
                         "sample": f"{W // 4}x{H // 4} px x 1 spp, {int(cnt1.sum())} paths in {dt1:.1f} s"}}


def _oracle_many_lights_worker(conn):
    """Spawned process: builds the oracle's scene of the many-light workload
    (not timed: about a minute, single-threaded), then waits for "go" and
    times a bounded sample, 1 spp over the full 1920 x 1080 image at depth 12,
    on all host cores."""
    import oracle
    from paper_1705_01263_gb300 import scenes as sc_mod
    sd, cam = sc_mod.instanced_field()
    t0 = time.time()
    osc = oracle.Scene(sd)
    build_s = time.time() - t0
    conn.send({"built": build_s})
    if conn.recv() != "go":
        return
    t0 = time.time()
    _, _, cnt, rays = osc.render(cam, 1, 12)
    dt = time.time() - t0
    paths = int(cnt.sum())
    conn.send({"value": paths / dt / 1e6, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"{cam.width}x{cam.height} px x 1 of the 256 spp (depth 12), {paths} paths in {dt:.1f} s; "
                         f"oracle scene build {build_s:.1f} s (flattened 10M triangles) not timed",
               "mrays_per_s": rays / dt / 1e6, "cpu": cpu_model()})


class OracleManyLights:
    """The many-light oracle sample in a process of its own, started with
    spawn before the first GPU call so that its scene build overlaps the GPU
    measurements; its timed render runs once they are done."""

    def __init__(self):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.conn, child = ctx.Pipe()
        self.proc = ctx.Process(target=_oracle_many_lights_worker, args=(child,), daemon=True)
        self.proc.start()

    def result(self, timeout=600):
        try:
            if not self.conn.poll(timeout):
                return None
            self.conn.recv()            # built
            self.conn.send("go")
            if not self.conn.poll(timeout):
                return None
            return self.conn.recv()
        finally:
            self.proc.join(1)
            if self.proc.is_alive():
                self.proc.terminate()

    def cancel(self):
        if self.proc.is_alive():
            self.proc.terminate()


def l2_peak(mb=16, reps=200):
    """Measured L2 copy bandwidth: a device-to-device copy of an `mb` MiB
    buffer (source and destination both resident in the 129 MB L2) repeated
    `reps` times, read + write bytes over the CUDA-event time (best of 3)."""
    import torch
    n = mb << 20
    a = torch.empty(n, dtype=torch.uint8, device="cuda")
    b = torch.empty_like(a)
    a.fill_(1)
    for _ in range(10):
        b.copy_(a)
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.copy_(a)
        e1.record()
        e1.synchronize()
        gbs = 2 * n * reps / (e0.elapsed_time(e1) / 1e3) / 1e9
        best = gbs if best is None else max(best, gbs)
    return best


def scheduler_sweep(scene, cam, spp, depth, pools=(1 << 22, 1 << 23, 1 << 24, 1 << 25)):
    """Regeneration (Sec. 3.1.3) against iteration sets on the benchmark
    workload: one timed render (CUDA events, L2 flushed before) per pool size
    with the paper's refill rule (half the pool ended), one with refills at
    every step, and the iteration-set scheduler holding the whole request."""
    import torch
    from paper_1705_01263_gb300 import rt
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    film = rt.Film(cam.width, cam.height)
    paths = cam.width * cam.height * spp

    def timed(**kw):
        film.clear()
        rt.rt_render(scene, cam, spp, depth, film, rt.make_opts(**kw))   # warm: allocations
        film.clear()
        flush.zero_()
        st = rt.rt_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rt.rt_render(scene, cam, spp, depth, film, rt.make_opts(stats=st, **kw))
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        return {"Mpaths_per_s": paths / ms / 1e3, "ms": ms, "regen_steps": st.regen_sets,
                "wavefront_steps": st.wavefront_steps}

    out = {"workload": f"{cam.width}x{cam.height}, {spp} spp, depth {depth}"}
    out["iteration_sets_whole_request"] = timed(scheduler=1)
    whole = out["iteration_sets_whole_request"]["Mpaths_per_s"]
    for p in pools:
        r = timed(max_paths=p)
        r["of_whole_request"] = r["Mpaths_per_s"] / whole
        out[f"regen_pool_{p >> 20}M"] = r
    r = timed(max_paths=1 << 24, regen_fraction=1e-6)
    r["of_whole_request"] = r["Mpaths_per_s"] / whole
    out["regen_pool_16M_every_step"] = r
    # state compression (Sec. 3.1.1) A/B: the whole request in one pool,
    # uncompressed against compressed; image difference as mean relative L1
    film.clear()
    rt.rt_render(scene, cam, spp, depth, film, rt.make_opts())
    ref = film.resolve()[0].double()
    for name, kw in (("uncompressed", {}), ("compressed", {"state_compression": True})):
        r = timed(**kw)
        r["of_whole_request"] = r["Mpaths_per_s"] / whole
        r["state_bytes_per_path"] = 132 if kw else 168
        img = film.resolve()[0].double()
        r["image_rel_l1_vs_uncompressed"] = float((img - ref).abs().sum() / ref.abs().sum())
        out[f"state_{name}"] = r
    film.close()
    return out


def many_lights_full(spp=256, depth=12):
    """The many-light configuration at its own size: 10M instanced triangles,
    100k textured emitters picked by the alias table, 1920 x 1080, 256 spp,
    depth 12 (530.8M paths), one timed render (CUDA events) after a warm-up
    render of 1 spp."""
    import torch
    from paper_1705_01263_gb300 import rt, scenes
    sd, cam = scenes.instanced_field()
    sd.light_bvh = False
    scene = rt.Scene(sd)
    film = rt.Film(cam.width, cam.height)
    rt.rt_render(scene, cam, 1, depth, film)
    film.clear()
    st = rt.rt_stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    rt.rt_render(scene, cam, spp, depth, film, rt.make_opts(stats=st))
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    out = {"workload": f"instanced field 10M tris (1000 instances of 100 meshes), 100k textured emitters, alias "
                       f"table, {cam.width}x{cam.height}, {spp} spp, depth {depth}",
           "paths": st.paths, "ms": ms, "Mpaths_per_s": st.paths / ms / 1e3,
           "Mrays_per_s": (st.extension_rays + st.shadow_rays) / ms / 1e3,
           "rays_per_path": (st.extension_rays + st.shadow_rays) / max(1, st.paths),
           "regen_steps": st.regen_sets, "wavefront_steps": st.wavefront_steps}
    film.close()
    del scene
    return out


def guided_vs_plain(light="down", target_spp=16384, chunk=512, max_factor=2, seed=5, guide_kw=None, opts_kw=None):
    """Time to equal RMSE, guided vs plain, on the Cornell configuration (64 x
    64, depth 8): light "down" is the configuration itself; "up" turns the
    emitter to face the ceiling, so that the room is lit through the bright
    patch it makes there; "door" lights the room from a closed side chamber
    through a door (the case a guide is for: from almost every visible point
    next-event estimation is blocked and a path must find the door; on "down"
    the pixel error is almost all direct light, which next-event estimation
    already samples). RMSE against the stored FP64 oracle reference (2^15 spp,
    2^17 for "door", from a disjoint part of the sample sequence) after every
    call of `chunk` spp; the target is the plain tracer's RMSE at
    `target_spp`; guided time includes its inference and training from an
    untrained network."""
    import torch
    from paper_1705_01263_gb300 import rt, scenes
    name = {"down": "cornell_64_depth8_ref.npz", "up": "cornell_up_64_depth8_ref.npz",
            "door": "cornell_door_64_depth8_ref.npz"}[light]
    ref_path = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(ref_path):
        return None
    ref_npz = np.load(ref_path)
    ref = ref_npz["mean"]
    sd, cam = scenes.door_room() if light == "door" else scenes.cornell_box(light=light)
    scene = rt.Scene(sd)
    mean = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")

    def curve(guided, stop_rmse=None, max_spp=target_spp):
        film = rt.Film(cam.width, cam.height)
        # warm-up of the code path on a scratch film (not timed)
        scratch = rt.Film(cam.width, cam.height)
        gk = guide_kw or {}
        rt.rt_render(scene, cam, chunk, 8, scratch,
                     rt.make_opts(guide=rt.Guide(scene, seed=seed + 1, **gk) if guided else None))
        torch.cuda.synchronize()
        guide = rt.Guide(scene, seed=seed, **gk) if guided else None
        pts = []
        t0 = time.perf_counter()
        spp = 0
        while spp < max_spp:
            rt.rt_render(scene, cam, chunk, 8, film, rt.make_opts(guide=guide, **((opts_kw or {}) if guided else {})))
            spp += chunk
            film.resolve(mean)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            img = mean.cpu().numpy().astype(np.float64)
            pts.append((spp, el, float(np.sqrt(np.mean((img - ref) ** 2)))))
            if stop_rmse is not None and pts[-1][2] <= stop_rmse:
                break
        return pts, guide

    plain, _ = curve(False)
    target = plain[-1][2]
    t_plain = plain[-1][1]
    guided, trained = curve(True, stop_rmse=target, max_spp=max_factor * target_spp)

    # per-sample gain of the network as trained by that run, frozen (no more
    # training steps): 2048 spp guided against 2048 spp plain on the same
    # iterations (2^19 on, disjoint from both curves and the reference)
    def frozen_rmse(g, spp=2048):
        f = rt.Film(cam.width, cam.height)
        f.seek(1 << 19)
        rt.rt_render(scene, cam, spp, 8, f, rt.make_opts(guide=g))
        f.resolve(mean)
        torch.cuda.synchronize()
        return float(np.sqrt(np.mean((mean.cpu().numpy().astype(np.float64) - ref) ** 2)))

    # (the first set of a call still runs one Adam step; at this learning
    # rate it moves no weight)
    frozen = rt.Guide(scene, seed=seed, train_every=1 << 30, lr=1e-30,
                      **{k: v for k, v in (guide_kw or {}).items() if k not in ("train_every", "lr")})
    frozen.load(trained.state())
    r_frozen, r_plain2k = frozen_rmse(frozen), frozen_rmse(None)
    t_guided, spp_guided = None, None
    for spp, el, r in guided:
        if r <= target:
            t_guided, spp_guided = el, spp
            break
    same = {p[0]: p[2] for p in plain}
    per_sample = [(spp, same[spp], r) for spp, _, r in guided if spp in same]
    # a short target as well: the plain tracer's RMSE at 256 spp (one
    # render of 256 spp, timed alike); guided reaches it within its first
    # call or later
    film = rt.Film(cam.width, cam.height)
    t0 = time.perf_counter()
    rt.rt_render(scene, cam, 256, 8, film, rt.make_opts())
    film.resolve(mean)
    torch.cuda.synchronize()
    t256 = time.perf_counter() - t0
    r256 = float(np.sqrt(np.mean((mean.cpu().numpy().astype(np.float64) - ref) ** 2)))
    g256 = next(((spp, el) for spp, el, r in guided if r <= r256), None)
    short = {"target_rmse": r256, "plain_seconds": t256, "plain_spp": 256,
             "guided_seconds": g256[1] if g256 else None, "guided_spp": g256[0] if g256 else None,
             "guided_speedup": (t256 / g256[1]) if g256 else None}
    where = {"down": "emitter under the ceiling facing down", "up": "emitter facing the ceiling",
             "door": "lit from a side chamber through a door"}[light]
    return {"scene": f"cornell 64x64, depth 8, {where}",
            "reference": f"FP64 oracle, {int(ref_npz['spp'])} spp from sequence iteration 2^20", "target_rmse": target,
            "target": f"plain RMSE at {target_spp} spp", "plain_seconds": t_plain, "plain_spp": plain[-1][0],
            "guided_seconds": t_guided, "guided_spp": spp_guided,
            "guided_speedup": (t_plain / t_guided) if t_guided else None,
            "rmse_at_equal_spp": per_sample[-4:], "target_256spp": short,
            "trained_guide_frozen_2048spp": {"guided_rmse": r_frozen, "plain_rmse": r_plain2k,
                                             "mse_gain": (r_plain2k / r_frozen) ** 2},
            "plain_curve": plain[::4], "guided_curve": guided[::4]}


def many_lights(spp=4, depth=12, ref_spp=128):
    """Secondary workload: 1000 instances of 100 meshes (10M instanced
    triangles), 100k textured emitters, 1920 x 1080 at `spp` of its 256 spp,
    depth 12. NEE picks emitters by the alias table and by the probabilistic
    light hierarchy (Sec. 2.1.1); for each, device time and paths/s, and the
    RMSE of the `spp` image against a `ref_spp` hierarchy reference of
    disjoint iterations. efficiency = (RMSE^2 x time) of the alias table over
    that of the hierarchy (above 1: the hierarchy reaches equal error
    sooner)."""
    import torch
    from paper_1705_01263_gb300 import rt, scenes
    sd, cam = scenes.instanced_field()
    film = rt.Film(cam.width, cam.height)

    def run(scene, first, n, stats=None):
        film.clear()
        film.seek(first)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        rt.rt_render(scene, cam, n, depth, film, rt.make_opts(stats=stats))
        ev1.record()
        ev1.synchronize()
        return film.resolve()[0], ev0.elapsed_time(ev1)

    out = {"workload": "instanced field: 1000 instances of 100 meshes, 10M instanced tris, 100k textured emitters, "
                       f"1920x1080, {spp} spp, depth {depth}; RMSE against {ref_spp} spp of disjoint iterations"}
    ref = None
    for name, bvh in (("light_hierarchy", True), ("alias_table", False)):
        sd.light_bvh = bvh
        s = rt.Scene(sd)
        if ref is None:
            ref, _ = run(s, 1 << 20, ref_spp)
            ref = ref.clone()
        run(s, 0, 1)   # warm-up
        st = rt.rt_stats()
        m, ms = run(s, 0, spp, st)
        info = s.info()
        out[name] = {"Mpaths_per_s": st.paths / ms / 1e3, "Mrays_per_s": (st.extension_rays + st.shadow_rays) / ms / 1e3,
                     "ms": ms, "rmse": float((m - ref).double().pow(2).mean().sqrt()),
                     "device_bytes": info["device_bytes"]}
        del s
    h, a = out["light_hierarchy"], out["alias_table"]
    out["efficiency"] = (a["rmse"] ** 2 * a["ms"]) / (h["rmse"] ** 2 * h["ms"])
    # direct light only (depth 1), where the choice of emitter is the whole
    # of the next-event estimate: same comparison at 4 spp
    direct, dref = {}, None
    for name, bvh in (("light_hierarchy", True), ("alias_table", False)):
        sd.light_bvh = bvh
        s = rt.Scene(sd)

        def run1(first, n):
            film.clear()
            film.seek(first)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            rt.rt_render(s, cam, n, 1, film)
            e1.record()
            e1.synchronize()
            return film.resolve()[0], e0.elapsed_time(e1)

        if dref is None:
            dref = run1(1 << 20, ref_spp)[0].clone()
        run1(0, 1)
        m, ms = run1(0, spp)
        direct[name] = {"rmse": float((m - dref).double().pow(2).mean().sqrt()), "ms": ms}
        del s
    dh, da = direct["light_hierarchy"], direct["alias_table"]
    direct["efficiency"] = (da["rmse"] ** 2 * da["ms"]) / (dh["rmse"] ** 2 * dh["ms"])
    out["direct_only"] = direct
    # irradiance probes (Sec. 4.2) among the instances, direct light only:
    # no emitter is seen directly, so the error is the next-event
    # estimate's alone
    n_side, pspp = 64, 16
    xs, zs = np.linspace(-26.0, 26.0, n_side), np.linspace(-43.0, 3.0, n_side)
    X, Z = np.meshgrid(xs, zs)
    pos = torch.from_numpy(np.stack([X.ravel(), np.full(X.size, 1.0), Z.ravel()], 1).astype(np.float32)).cuda()
    nrm = torch.from_numpy(np.tile(np.array([[0.0, 1.0, 0.0]], np.float32), (X.size, 1))).cuda()
    pfilm = rt.Film(X.size, 1)
    probes_out, pref = {}, None
    for name, bvh in (("light_hierarchy", True), ("alias_table", False)):
        sd.light_bvh = bvh
        s = rt.Scene(sd)

        def runp(first, n):
            pfilm.clear()
            pfilm.seek(first)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            rt.rt_render_probes(s, pos, nrm, n, 1, pfilm)
            e1.record()
            e1.synchronize()
            return pfilm.resolve()[0], e0.elapsed_time(e1)

        if pref is None:
            pref = runp(1 << 20, 64 * pspp)[0].clone()
        runp(0, 1)
        m, ms = runp(0, pspp)
        probes_out[name] = {"rmse": float((m - pref).double().pow(2).mean().sqrt()), "ms": ms}
        del s
    ph, pa = probes_out["light_hierarchy"], probes_out["alias_table"]
    probes_out["efficiency"] = (pa["rmse"] ** 2 * pa["ms"]) / (ph["rmse"] ** 2 * ph["ms"])
    probes_out["workload"] = f"{X.size} probes at height 1 among the instances, normals up, direct light, {pspp} spp"
    out["probes_direct"] = probes_out
    pfilm.close()
    out["bvh_nodes"], out["unique_tris"] = info["nodes"], info["leaf_tris"]
    film.close()
    return out


def batched(spp_divisor=16):
    """Secondary workload: 64 independent seeded scenes (1k-500k triangles,
    256^2-1024^2 px, depth 4-16, spp drawn from 16..256 and divided by
    `spp_divisor` to bound the run) in one batched wavefront replayed as a
    CUDA graph; pool capacity chosen by the autotuner on 1 spp per job."""
    import torch
    from paper_1705_01263_gb300 import rt, scenes
    t0 = time.time()
    specs = scenes.batch_jobs(spp_divisor=spp_divisor)
    built = [(rt.Scene(sd), cam, spp, d) for sd, cam, spp, d in specs]
    films = [rt.Film(cam.width, cam.height) for _, cam, _, _ in built]
    jobs = [(s, cam, spp, d, f) for (s, cam, spp, d), f in zip(built, films)]
    setup_s = time.time() - t0
    o = rt.rt_autotune(jobs, 1)
    for f in films:
        f.clear()
    st = rt.rt_stats()
    o.stats = C_pointer(st)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    rt.rt_render_batch(jobs, o)
    ev1.record()
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    # the same batch with a guiding network on every 8th job and on every
    # job (each trained from scratch during the call): one shared wavefront
    # over the jobs' tasks interleaved image by image, sets of 2^23 paths, one
    # network launch per job and guided bounce step, 8 warm-up steps (one
    # after each set), then one step per 2^20 of the job's paths (every 4th
    # such step taken)
    with_guides = {}
    for every in (8, 1):
        for f in films:
            f.clear()
        guides = [rt.Guide(s, seed=7 + k, warm_steps=8, train_every=4) if k % every == 0 else None
                  for k, (s, _, _, _, _) in enumerate(jobs)]
        gjobs = [j + (g,) for j, g in zip(jobs, guides)]
        go = rt.make_opts(tail_threshold=o.tail_threshold, trace_kernel=o.trace_kernel, block_size=o.block_size)
        gst = rt.rt_stats()
        go.stats = C_pointer(gst)
        torch.cuda.synchronize()
        ev0.record()
        rt.rt_render_batch(gjobs, go)
        ev1.record()
        ev1.synchronize()
        gms = ev0.elapsed_time(ev1)
        for g in guides:
            if g is not None:
                g.close()
        n_g = sum(g is not None for g in guides)
        with_guides[f"{n_g}_of_64"] = {"guided_jobs": n_g, "ms": gms, "Mpaths_per_s": gst.paths / gms / 1e3,
                                       "sets": gst.waves, "kernel_launches": gst.kernel_launches}
    return {"workload": f"64 seeded scenes ({sum(sd.num_triangles for sd, _, _, _ in specs)} triangles in all), "
                        f"spp / {spp_divisor}, one batched wavefront replayed as a CUDA graph",
            "paths": st.paths, "Mpaths_per_s": st.paths / ms / 1e3,
            "Mrays_per_s": (st.extension_rays + st.shadow_rays) / ms / 1e3, "ms": ms,
            "graph_replays": st.waves, "autotuned_pool": o.max_paths_in_flight, "autotuned_block": o.block_size,
            "scene_setup_s": setup_s,
            "with_guides": with_guides}


def traversal_only(sd, cam, scene, n=1 << 22, reps=5):
    """Traversal-only throughput through rt_trace on synthetic ray batches of
    the main scene, 2^22 rays each: camera rays in scanline order (coherent,
    closest hit), rays leaving random surface points in uniform directions
    (incoherent, standing in for diffuse bounces, closest hit) and segments
    between two surface points (shadow rays, any hit). Device time per batch
    with CUDA events, L2 flushed between batches; median of `reps`."""
    import torch
    from paper_1705_01263_gb300 import rt, scenes
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for name, kind, seed, any_hit in (("camera", "camera", 31, False), ("diffuse", "incoherent", 32, False),
                                      ("shadow", "shadow", 33, True)):
        rays = torch.from_numpy(scenes.random_rays(sd, n, seed, kind, cam)).cuda()
        hits, soa = rt.rt_trace(scene, rays, any_hit)
        torch.cuda.synchronize()
        ms = []
        for _ in range(2 + reps):
            flush.zero_()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            rt.rt_trace(scene, soa, any_hit, hits=hits)
            ev1.record()
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        med = statistics.median(ms[2:])
        out[name] = {"rays": n, "any_hit": any_hit, "ms": med, "Mrays_per_s": n / med / 1e3,
                     "hit_fraction": float((hits[0] != -1).float().mean().item())}
        del rays, soa, hits
    return out


def probes(sd, scene, n_side=64, spp=256, depth=16):
    """Irradiance probes (Sec. 4.2) in the main scene: an n_side x n_side grid
    over the middle half of the scene at a fifth of its height (between and
    through the spheres, like a grid of probes at desk height in a room),
    normals up, `spp` samples each, depth 16 (device time, Mpaths/s)."""
    import torch
    from paper_1705_01263_gb300 import rt
    V = sd.vertices
    lo, hi = V.min(0), V.max(0)
    xs = np.linspace(lo[0] + 0.25 * (hi[0] - lo[0]), hi[0] - 0.25 * (hi[0] - lo[0]), n_side)
    zs = np.linspace(lo[2] + 0.25 * (hi[2] - lo[2]), hi[2] - 0.25 * (hi[2] - lo[2]), n_side)
    X, Z = np.meshgrid(xs, zs)
    y = lo[1] + 0.2 * (hi[1] - lo[1])
    pos = np.stack([X.ravel(), np.full(X.size, y), Z.ravel()], 1).astype(np.float32)
    nrm = np.tile(np.array([[0.0, 1.0, 0.0]], np.float32), (X.size, 1))
    pd, nd = torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda()
    film = rt.Film(X.size, 1)
    rt.rt_render_probes(scene, pd, nd, 4, depth, film)
    torch.cuda.synchronize()
    st = rt.rt_stats()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    rt.rt_render_probes(scene, pd, nd, spp, depth, film, rt.make_opts(stats=st))
    ev1.record()
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    mean = torch.empty((1, X.size, 3), dtype=torch.float32, device="cuda")
    film.resolve(mean)
    E = mean.cpu().numpy()
    return {"workload": f"{X.size} irradiance probes (grid over the ground, normals up), {spp} spp, depth {depth}",
            "Mpaths_per_s": st.paths / ms / 1e3, "Mrays_per_s": (st.extension_rays + st.shadow_rays) / ms / 1e3,
            "ms": ms, "irradiance_mean_rgb": [float(x) for x in E.reshape(-1, 3).mean(0)]}


def env_normal_vs_plain(sd, cam, scene, spp=16, ref_spp=1024, reps=3):
    """Environment NEE through the normal-oriented top pyramid levels (Sec.
    2.1.2; the default) against the plain pyramid (env_plain) in the main
    scene at equal spp: RMSE of `spp`-sample images against a `ref_spp`
    reference of disjoint iterations, and device time per image. efficiency
    = (RMSE^2 x time) of plain over that of normal-oriented (above 1: the
    normal-oriented levels reach equal error sooner)."""
    import dataclasses
    import torch
    from paper_1705_01263_gb300 import rt
    plain = rt.Scene(dataclasses.replace(sd, env_plain=True))
    film = rt.Film(cam.width, cam.height)

    def render(sc, first, n):
        film.clear()
        film.seek(first)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        rt.rt_render(sc, cam, n, DEPTH, film)
        ev1.record()
        ev1.synchronize()
        mean, _ = film.resolve()
        return mean, ev0.elapsed_time(ev1)

    ref, _ = render(scene, 1 << 22, ref_spp)
    out = {"workload": f"{WORKLOAD.replace('64 spp', f'{spp} spp')}, reference {ref_spp} spp of disjoint iterations"}
    for name, sc in (("normal_oriented", scene), ("plain", plain)):
        render(sc, 0, spp)   # warm-up
        err, ms = [], []
        for r in range(reps):
            m, t = render(sc, r * spp, spp)
            err.append(float((m - ref).double().pow(2).mean().sqrt()))
            ms.append(t)
        out[name] = {"rmse": statistics.mean(err), "ms": statistics.median(ms)}
    n, p = out["normal_oriented"], out["plain"]
    out["efficiency"] = (p["rmse"] ** 2 * p["ms"]) / (n["rmse"] ** 2 * n["ms"])
    film.close()
    del plain
    return out


def two_way_vs_plain(res=256, depth=4, spp=64, ref_spp=4096, reps=3, scene_name="glossy"):
    """Two-way path tracing (Sec. 2: the light tracer as a third MIS
    technique, rt_render_two_way) against the path tracer (rt_render) in the
    glossy room lit through its ceiling, at equal iterations: RMSE against a
    two-way reference of `ref_spp` disjoint iterations and device time.
    efficiency = (RMSE^2 x time) of the path tracer over two-way's (above 1:
    two-way reaches equal error sooner)."""
    import torch
    from paper_1705_01263_gb300 import rt, scenes
    if scene_name == "glossy":
        sd, cam = scenes.glossy_room(res)
        what = f"glossy room lit through its ceiling, {res}x{res}"
    elif scene_name == "turntable":
        # a near-mirror sphere on a stand close to the camera in an open,
        # sky-lit scene a few hundred times larger (Sec. 2.1.3's setting)
        sd, cam = scenes.turntable(res)
        what = f"turntable (near-mirror sphere, open sky-lit scene), {res}x{res}"
    else:
        # the main scene, open and lit by the sky
        sd, cam = scenes.sphere_field()
        cam.width, cam.height = 2 * res, res
        what = f"sphere field (sky-lit, open), {2 * res}x{res}"
    scene = rt.Scene(sd)
    film = rt.Film(cam.width, cam.height)
    npix = cam.width * cam.height

    def timed(fn):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        r = fn()
        ev1.record()
        ev1.synchronize()
        return r, ev0.elapsed_time(ev1)

    def plain(first, n):
        film.clear()
        film.seek(first)
        _, ms = timed(lambda: rt.rt_render(scene, cam, n, depth, film))
        mean, _ = film.resolve()
        return mean, ms, None

    def two_way(first, n, lt_emission=0, lt_mode=0):
        film.clear()
        film.seek(first)
        o = rt.make_opts(lt_emission=lt_emission)
        st, ms = timed(lambda: rt.rt_render_two_way(scene, cam, n, depth, film, o, lt_mode=lt_mode))
        mean, _ = film.resolve()
        return mean, ms, st

    ref, _, _ = two_way(1 << 22, ref_spp)
    out = {"workload": f"{what}, depth {depth}, {spp} iterations; reference: two-way, {ref_spp} disjoint iterations"}
    runs = (("path_tracer", plain), ("two_way", two_way),
            ("two_way_uniform_emission", lambda f, n: two_way(f, n, lt_emission=1)),
            ("light_tracer_alone_aimed", lambda f, n: two_way(f, n, lt_mode=1)),
            ("light_tracer_alone_uniform", lambda f, n: two_way(f, n, lt_emission=1, lt_mode=1)))
    for name, fn in runs:
        fn(0, spp)   # warm-up
        err, ms = [], []
        st = None
        for r in range(reps):
            m, t, st = fn(r * spp, spp)
            err.append(float((m - ref).double().pow(2).mean().sqrt()))
            ms.append(t)
        out[name] = {"rmse": statistics.mean(err), "ms": statistics.median(ms)}
        if st is not None:
            paths = 2 * spp * npix   # camera paths + light paths
            out[name].update({"Mpaths_per_s": paths / (out[name]["ms"] / 1e3) / 1e6,
                              "Mrays_per_s": (st.extension_rays + st.shadow_rays) / (out[name]["ms"] / 1e3) / 1e6})
        else:
            out[name]["Mpaths_per_s"] = spp * npix / (out[name]["ms"] / 1e3) / 1e6
    p_, t_, u_ = out["path_tracer"], out["two_way"], out["two_way_uniform_emission"]
    out["rmse_ratio"] = t_["rmse"] / p_["rmse"]
    out["efficiency"] = (p_["rmse"] ** 2 * p_["ms"]) / (t_["rmse"] ** 2 * t_["ms"])
    # photon aiming (Sec. 2.1.3) against uniform emission, with MIS and for
    # the light tracer alone (where the emission decides the error)
    out["aiming_efficiency"] = (u_["rmse"] ** 2 * u_["ms"]) / (t_["rmse"] ** 2 * t_["ms"])
    la, lu = out["light_tracer_alone_aimed"], out["light_tracer_alone_uniform"]
    out["aiming_efficiency_light_tracer_alone"] = (lu["rmse"] ** 2 * lu["ms"]) / (la["rmse"] ** 2 * la["ms"])
    film.close()
    return out


# FLOPs of one row of the guiding network: 224->64->64->64->64->40
GUIDE_FLOP_PER_ROW = 2 * (224 * 64 + 3 * 64 * 64 + 64 * 40)


def guide_mlp(n=1 << 20, reps=10):
    """Guiding-network throughput on the tensor cores: the fused inference
    kernel through rt_guide_infer on n rows of uniform features already on
    the device (median of `reps`, CUDA events, L2 flushed between calls),
    against the measured dense BF16 peak; and one fused training step
    (forward with the loss gradient, backward, Adam) on 2^16 samples."""
    import torch
    from paper_1705_01263_gb300 import rt
    hbm, tflops, src = peaks()
    g = rt.Guide(None, seed=3)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    feat = torch.rand((n, 7), device="cuda", generator=gen)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    raw = g.infer(feat)
    torch.cuda.synchronize()
    # the kernel alone: rt_guide_infer_async between the events (the
    # synchronous call would add its host round trip for the status), the
    # status checked after each timed launch
    ms, ms_sync = [], []
    for _ in range(reps):
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        g.infer_async(feat, raw)
        ev1.record()
        ev1.synchronize()
        g.check()
        ms.append(ev0.elapsed_time(ev1))
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        g.infer(feat)
        ev1.record()
        ev1.synchronize()
        ms_sync.append(ev0.elapsed_time(ev1))
    med = statistics.median(ms)
    achieved = GUIDE_FLOP_PER_ROW * n / med / 1e9
    m = 1 << 16
    wi = torch.nn.functional.normalize(torch.randn((m, 3), device="cuda", generator=gen), dim=1)
    wt = torch.rand(m, device="cuda", generator=gen)
    g.train_step(feat[:m], wi, wt)
    torch.cuda.synchronize()
    tms = []
    for _ in range(reps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        g.train_step(feat[:m], wi, wt)
        ev1.record()
        ev1.synchronize()
        tms.append(ev0.elapsed_time(ev1))
    g.close()
    return {"workload": f"fused inference of {n} rows (224-64-64-64-64-40, BF16 weights, FP32 accumulation)",
            "kernel": "k_guide_mlp (tcgen05)", "ms": med, "Mrows_per_s": n / med / 1e3,
            "ms_synchronous_call": statistics.median(ms_sync),
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": tflops, "unit": "TFLOP/s",
                         "frac": achieved / tflops, "flop_per_row": GUIDE_FLOP_PER_ROW,
                         "peak_source": f"{src} bf16_tflops (burst)"},
            "train_step_ms_65536": statistics.median(tms)}


def C_pointer(x):
    import ctypes
    return ctypes.pointer(x)


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    from paper_1705_01263_gb300 import scenes
    sd, cam = scenes.sphere_field()
    import oracle
    osc = oracle.Scene(sd)
    # each timed step: the workload's own image (1920 x 1080) at one of its
    # 64 iterations (about 2 s on 16 cores); warm-up steps on a small crop
    W, H = cam.width, cam.height
    c2 = scenes.Camera(cam.eye, cam.look_at, cam.up, cam.vfov_deg, W, H)
    cw = scenes.Camera(cam.eye, cam.look_at, cam.up, cam.vfov_deg, 240, 135)
    for _ in range(args.warmup):
        osc.render(cw, 1, DEPTH)
    times, paths = [], 0
    for k in range(args.steps):
        t0 = time.time()
        _, _, cnt, _ = osc.render(c2, 1, DEPTH, iter0=k % SPP)
        times.append(time.time() - t0)
        paths += int(cnt.sum())
    total = sum(times)
    v = paths / total / 1e6
    cores = os.cpu_count() or 1
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "reference_sample": f"{W}x{H} px, 1 of the {SPP} spp per step"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                             "sample": f"{W}x{H} px x 1 spp per step of the same scene/camera, depth {DEPTH}"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-guided", action="store_true", help="skip the guided-vs-plain time-to-RMSE run")
    ap.add_argument("--guided-once", default="", help="only the guided-vs-plain comparison on these scenes "
                    "(comma-separated: up, down, door), printed one line each")
    ap.add_argument("--no-many-lights", action="store_true", help="skip the instanced many-light workload")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-scene batched workload")
    ap.add_argument("--no-two-way", action="store_true", help="skip the two-way against path-tracer comparison")
    ap.add_argument("--two-way-once", action="store_true", help="only the two-way comparison (for profiling)")
    ap.add_argument("--tw-spp", type=int, default=64, help="iterations per image of --two-way-once")
    ap.add_argument("--tw-ref-spp", type=int, default=4096, help="reference iterations of --two-way-once")
    ap.add_argument("--tw-scene", default="all", choices=["all", "glossy", "spheres", "turntable"],
                    help="scene of --two-way-once")
    ap.add_argument("--no-traversal", action="store_true", help="skip the traversal-only ray batches")
    ap.add_argument("--no-probes", action="store_true", help="skip the irradiance-probe workload")
    ap.add_argument("--mlp-once", action="store_true",
                    help="run only the guiding-network throughput measurement and print it (profile captures)")
    ap.add_argument("--no-env-ab", action="store_true",
                    help="skip the normal-oriented vs plain environment-sampling comparison")
    ap.add_argument("--pool", type=int, default=0, help="paths in flight per iteration set (0 = library default)")
    ap.add_argument("--tail", type=int, default=0, help="live-path count below which the megakernel finishes a set (0 = default)")
    ap.add_argument("--render-once", action="store_true",
                    help="profiling aid: one untimed render of --spp, print its ray and launch counts, exit")
    ap.add_argument("--scene", default="field", choices=["field", "cornell", "cornell-up", "many-lights"],
                    help="scene of --render-once (cornell-up: emitter facing the ceiling; many-lights: the "
                         "instanced 100k-emitter field with the light hierarchy, depth 12)")
    ap.add_argument("--guided", action="store_true",
                    help="--render-once with the guiding network: three calls of --spp (the first trains it)")
    ap.add_argument("--spp", type=int, default=SPP)
    ap.add_argument("--out", default=None)
    ap.add_argument("--trace-kernel", type=int, default=0,
                    help="0 closest hit one ray per thread with warp fetch, shadow rays with lane refill; "
                         "1 persistent warps refilling lanes; 2 one ray per thread with a shared-memory stack; "
                         "3 lane refill between node visits for both; 4 one ray per thread for both; "
                         "5 as 0 for camera rays, as 3 for later bounces; 6 closest hit one ray per thread with "
                         "postponed triangle tests, shadow rays as 0; 7 postponed triangle tests for both; 8 closest hit with "
                         "per-child stack entries, nearest child next, far entries dropped on pop")
    ap.add_argument("--megakernel-only", action="store_true", help="A/B baseline: megakernel per iteration set")
    ap.add_argument("--sort-by-material", action="store_true", help="A/B: material-sorted shading queue")
    ap.add_argument("--sort-rays", action="store_true", help="A/B: reorder extension rays by octant and origin cell")
    ap.add_argument("--scheduler", type=int, default=0, help="0 regeneration (default), 1 iteration sets")
    ap.add_argument("--regen-fraction", type=float, default=0.0, help="refill once this fraction ended (0 = 0.5)")
    ap.add_argument("--no-scheduler-sweep", action="store_true", help="skip the regeneration pool-size sweep")
    ap.add_argument("--no-many-lights-full", action="store_true",
                    help="skip the many-light configuration at its own size (256 spp) and its oracle sample")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = env_rank()
    quick = args.render_once or args.mlp_once or args.two_way_once
    # the many-light oracle sample: spawned before the first GPU call, its
    # scene build overlaps the GPU measurements
    oml = None
    if rank == 0 and world == 1 and not quick and not args.no_cpu_baseline and not args.no_many_lights_full:
        oml = OracleManyLights()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1705_01263_gb300 import rt, scenes
    rt.lib()
    sd, cam = scenes.sphere_field()
    scene = rt.Scene(sd)
    film = rt.Film(cam.width, cam.height)
    stream = torch.cuda.current_stream()
    # each rank renders a disjoint iteration range: rank r starts at pass r * 10^6
    base_iter = rank * 1_000_000
    l2_flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    WH = cam.width * cam.height

    def opts(**kw):
        return rt.make_opts(seed=0, trace_kernel=args.trace_kernel, megakernel_only=args.megakernel_only,
                            sort_by_material=args.sort_by_material, sort_rays=args.sort_rays,
                            max_paths=args.pool, tail_threshold=args.tail, scheduler=args.scheduler,
                            regen_fraction=args.regen_fraction, **kw)

    def render_step(stats=None, profile=0):
        o = opts(stats=stats, profile=profile)
        rt.rt_render(scene, cam, args.spp, DEPTH, film, o)

    film.seek(base_iter)
    if args.mlp_once:
        print(json.dumps(guide_mlp(reps=3)), flush=True)
        return 0
    if args.guided_once:
        for light in args.guided_once.split(","):
            print(json.dumps({"light": light, **(guided_vs_plain(light) or {})}), flush=True)
        return 0
    if args.two_way_once:
        if args.tw_scene in ("all", "glossy"):
            print(json.dumps(two_way_vs_plain(spp=args.tw_spp, ref_spp=args.tw_ref_spp, reps=1)), flush=True)
        if args.tw_scene in ("all", "spheres"):
            print(json.dumps(two_way_vs_plain(res=270, depth=8, spp=16, ref_spp=256, reps=1, scene_name="spheres")),
                  flush=True)
        if args.tw_scene in ("all", "turntable"):
            print(json.dumps(two_way_vs_plain(res=128, depth=4, spp=args.tw_spp, ref_spp=args.tw_ref_spp, reps=1,
                                              scene_name="turntable")), flush=True)
        return 0
    if args.render_once:
        st = rt.rt_stats()
        what = WORKLOAD.replace("64 spp", f"{args.spp} spp")
        if args.scene == "many-lights":
            msd, mcam = scenes.instanced_field()
            msd.light_bvh = True
            mscene = rt.Scene(msd)
            mfilm = rt.Film(mcam.width, mcam.height)
            rt.rt_render(mscene, mcam, args.spp, 12, mfilm, rt.make_opts(stats=st))
            what = f"many-lights 1920x1080 (light hierarchy), {args.spp} spp, depth 12"
        elif args.scene != "field" or args.guided:
            csd, ccam = scenes.cornell_box(light="up" if args.scene == "cornell-up" else "down")
            cscene = rt.Scene(csd)
            cfilm = rt.Film(ccam.width, ccam.height)
            guide = rt.Guide(cscene, seed=5) if args.guided else None
            for _ in range(3 if args.guided else 1):
                rt.rt_render(cscene, ccam, args.spp, 8, cfilm, rt.make_opts(guide=guide, stats=st))
            what = f"{args.scene} 64x64, {args.spp} spp, depth 8" + (", guided, 3 calls" if args.guided else "")
        else:
            render_step(st)
        torch.cuda.synchronize()
        print(json.dumps({"render_once": what, "paths": st.paths,
                          "extension_rays": st.extension_rays, "shadow_rays": st.shadow_rays,
                          "trace_launches": st.trace_launches, "wavefront_steps": st.wavefront_steps}), flush=True)
        return 0
    for _ in range(args.warmup):
        render_step()
    torch.cuda.synchronize()
    # instrumented pass (not timed): traversal work per ray for the roofline
    wstats = rt.rt_stats()
    render_step(wstats, profile=2)
    torch.cuda.synchronize()
    # timed steps: device time per step with CUDA events on the render stream,
    # L2 flushed between steps (outside the events)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, stats_list = [], []
    with ClockSampler(local) as clk:
        t_wall0 = time.time()
        for k in range(args.steps):
            l2_flush.zero_()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s = rt.rt_stats()
            ev0.record(stream)
            rt.rt_render(scene, cam, args.spp, DEPTH, film, opts(stats=s, profile=1))
            ev1.record(stream)
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
            stats_list.append(s)
        torch.cuda.synchronize()
        t_wall = time.time() - t_wall0
    if dist:
        dist.barrier()
    tot_ms = sum(step_ms)
    if dist:
        t = torch.tensor([tot_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    paths_per_step = WH * args.spp
    value = paths_per_step * args.steps * world / (tot_ms / 1e3) / 1e6
    ext = sum(s.extension_rays for s in stats_list)
    shd = sum(s.shadow_rays for s in stats_list)
    mrays = (ext + shd) * world / (tot_ms / 1e3) / 1e6
    launches = sum(s.kernel_launches for s in stats_list)
    # roofline of the dominant kernel (closest-hit traversal)
    trace_ms = sum(s.trace_ms for s in stats_list)
    tl = sum(s.trace_launches for s in stats_list)
    ext_rays_timed = ext
    nodes_per_ray = wstats.ext_nodes / max(1, wstats.extension_rays)
    tris_per_ray = wstats.ext_tris / max(1, wstats.extension_rays)
    # algorithmic bytes per extension ray: node visits x 80 B + triangle tests
    # x 36 B (three FP32 vertices) + 32 B ray in + 20 B hit out; the stored
    # triangle record is 48 B (vertices padded to float4, id in the pad)
    bytes_per_ray = nodes_per_ray * 80 + tris_per_ray * 36 + 32 + 20
    bytes_per_ray_stored = nodes_per_ray * 80 + tris_per_ray * 48 + 32 + 20
    # per launch: bytes of all rays of all launches / their total device time
    achieved_gbs = ext_rays_timed * bytes_per_ray / (trace_ms / 1e3) / 1e9 if trace_ms > 0 else None
    hbm, bf16, peak_src = peaks()
    shares = {"trace_ext": sum(s.trace_ms for s in stats_list), "shade": sum(s.shade_ms for s in stats_list),
              "trace_shadow": sum(s.shadow_ms for s in stats_list),
              "megakernel": sum(s.megakernel_ms for s in stats_list), "other": sum(s.other_ms for s in stats_list)}
    # end to end through the public API with host buffers: camera in, image out
    mean_dev = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    host_img = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, pin_memory=True)
    cam_bytes = 48
    torch.cuda.synchronize()
    e2e_ms = []
    for k in range(max(2, args.steps // 2)):
        l2_flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rt.rt_render(scene, cam, args.spp, DEPTH, film, opts())
        film.resolve(mean_dev)
        host_img.copy_(mean_dev, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_value = paths_per_step * world / (statistics.mean(e2e_ms) / 1e3) / 1e6
    gvp = None
    if rank == 0 and not args.no_guided:
        gvp = {"indirect_lit": guided_vs_plain("up"), "config": guided_vs_plain("down"),
               "door": guided_vs_plain("door")}
        # the same comparison with the network guiding only the first one or
        # two vertices, 8 warm-up steps and training after every 4th set
        variants = []
        for gd in (1, 2):
            kw = dict(guide_depth=gd, warm_steps=8, train_every=4)
            for key, light in (("indirect_lit", "up"), ("config", "down")):
                r = guided_vs_plain(light, guide_kw=kw)
                if r:
                    variants.append({"scene": key, **kw, "guided_speedup": r["guided_speedup"],
                                     "guided_spp": r["guided_spp"], "plain_spp": r["plain_spp"]})
        gvp["variants"] = variants
    ml = None
    if rank == 0 and not args.no_many_lights:
        ml = many_lights()
    trv = None
    if rank == 0 and not args.no_traversal:
        trv = traversal_only(sd, cam, scene)
    prb = None
    if rank == 0 and not args.no_probes:
        prb = probes(sd, scene)
    gmlp = None
    if rank == 0 and not args.no_guided:
        gmlp = guide_mlp()
    env_ab = None
    if rank == 0 and not args.no_env_ab:
        env_ab = env_normal_vs_plain(sd, cam, scene)
    bt = None
    if rank == 0 and not args.no_batched:
        bt = batched()
    tw = None
    if rank == 0 and not args.no_two_way:
        tw = two_way_vs_plain()
        tw["open_scene"] = two_way_vs_plain(res=270, depth=8, spp=16, ref_spp=256, scene_name="spheres")
        tw["turntable"] = two_way_vs_plain(res=128, depth=4, spp=64, ref_spp=4096, scene_name="turntable")
    sweep = None
    if rank == 0 and not args.no_scheduler_sweep:
        sweep = scheduler_sweep(scene, cam, args.spp, DEPTH)
    mlf = None
    if rank == 0 and not args.no_many_lights_full:
        mlf = many_lights_full()
    l2 = l2_peak() if rank == 0 else None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_oracle(sd, cam)
        if oml is not None and mlf is not None:
            mlf["cpu_baseline"] = oml.result()
    if oml is not None:
        oml.cancel()
    clocks = clk.summary()
    if rank == 0:
        achieved_l2 = (achieved_gbs / l2) if (achieved_gbs and l2) else None
        summary = {
            "mrays_per_s": mrays,
            "trace_ext_frac_hbm": (achieved_gbs / hbm) if achieved_gbs else None,
            "trace_ext_frac_l2": achieved_l2,
            "guided_speedup": {k: (gvp[k] or {}).get("guided_speedup") for k in ("indirect_lit", "config", "door")}
            if gvp else None,
            "guide_mlp_frac_bf16": gmlp["roofline"]["frac"] if gmlp else None,
            "many_lights_full_Mpaths_per_s": mlf["Mpaths_per_s"] if mlf else None,
            "regen_vs_whole_request": {k: v.get("of_whole_request") for k, v in sweep.items()
                                       if isinstance(v, dict) and "of_whole_request" in v} if sweep else None,
        }
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded generators; the paper's scenes are not available)",
            "config": {"workload": WORKLOAD, "triangles": sd.num_triangles, "width": cam.width,
                       "height": cam.height, "spp": args.spp, "max_depth": DEPTH,
                       "paths_per_step": paths_per_step, "l2": "flushed between steps (256 MiB write)",
                       "film": "FP64 sums", "parallelism": f"weak: {world} rank(s), disjoint iteration ranges",
                       "scheduler": ["regeneration (Sec. 3.1.3)", "iteration sets"][args.scheduler],
                       "pool": args.pool or "library default",
                       "trace_kernel": ["closest hit one ray per thread, shadow rays with lane refill",
                                        "persistent warps, lane refill",
                                        "one ray per thread, shared-memory stack",
                                        "lane refill between node visits", "one ray per thread",
                                        "camera rays one per thread, later bounces with lane refill",
                                        "closest hit one ray per thread with postponed triangle tests, "
                                        "shadow rays with lane refill",
                                        "one ray per thread with postponed triangle tests",
                                        "closest hit one ray per thread, nearest child next, far stack entries "
                                        "dropped"][args.trace_kernel],
                       "ray_order": "octant + origin cell" if args.sort_rays else "compaction order",
                       "schedule": "megakernel only" if args.megakernel_only else "wavefront + megakernel tail",
                       "shading_queue": "material-sorted" if args.sort_by_material else "compaction order"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": cam_bytes,
                    "d2h_bytes_per_step": cam.width * cam.height * 3 * 4},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "kernel": "k_trace_ext (closest-hit BVH8 traversal)",
                         "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                         "frac": (achieved_gbs / hbm) if achieved_gbs else None,
                         "traffic": TRACE_EXT_DRAM_BYTES_PER_RAY * ext_rays_timed / max(1, tl),
                         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per extension ray "
                                           "(4-spp capture) x rays per timed launch",
                         "peak_source": f"{peak_src} hbm_gbs",
                         "l2_peak": l2, "l2_frac": achieved_l2,
                         "l2_peak_source": "measured here: 16 MiB device-to-device copy, L2-resident",
                         "bytes_per_ray": bytes_per_ray, "bytes_per_ray_stored_layout": bytes_per_ray_stored,
                         "nodes_per_ray": nodes_per_ray,
                         "tris_per_ray": tris_per_ray, "launches": tl,
                         "avg_launch_ms": trace_ms / max(1, tl)},
            "cpu_baseline": cpu,
            "clocks": clocks,
            "summary": summary,
            "kernel_ms_share": {k: v / max(1e-9, sum(shares.values())) for k, v in shares.items()},
            "rays_per_path": (ext + shd) / (paths_per_step * args.steps),
            "many_lights_full": mlf,
            "scheduler_sweep": sweep,
            "guided_vs_plain": gvp,
            "guide_mlp": gmlp,
            "many_lights": ml,
            "batched": bt,
            "traversal_only": trv,
            "probes": prb,
            "env_normal_vs_plain": env_ab,
            "two_way": tw,
            "wall_s": t_wall,
        }
        s = json.dumps(line)
        print(s, flush=True)
        if args.out:
            with open(args.out, "w") as f:
                f.write(s + "\n")
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
