#!/usr/bin/env python
"""Proximal iterations per second of the GNRHTC ADMM step (Alg. 5, pure-L)
on a seeded synthetic 200x200x20x20 FP32 workload (400 DCT-transformed face
slices of rank 10, sigma = 1e-3 noise, 5% U(-1,1) outliers, 30% observed;
sketch width 20 = rank 10 + oversampling 10, one power iteration).

One "step" is one tr_prox_step: tube forward pass, the randomized prox of all
400 transformed slices, tube inverse pass.  The device-resident state
(L, E, Y, Lambda, G, Abar, Gbar: 7 x 64 MB) is far larger than the 129 MB L2,
so every step streams from HBM without an explicit flush.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

N > 1 (launched by torchrun): every rank runs an independent replica of the
workload (the method has no cross-problem exchange), scaling "weak".
"""

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "prox iters/s at rel-err<=1e-4 vs FP64 oracle; chosen vs plain form speedup"
UNIT = "iters/s"
WORKLOAD = "tubal200x400_r10"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-engine", default="rsvd", choices=["rsvd", "full"],
                    help=argparse.SUPPRESS)
    ap.add_argument("--prec", default="bf16x3", choices=["fp32", "bf16", "bf16x3"],
                    help="precision of the chosen form's slice products (default: split "
                         "BF16, the form whose stated bound is the metric's 1e-4)")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-width A/B on the power-law workload")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batch of 64 uneven problems")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the precision forms on the 1024x1024x64 workload")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the 64x64x16 FP64 workload")
    ap.add_argument("--no-tucker", action="store_true",
                    help="skip the shared-Tucker prox (Alg. 1 + Alg. 4) timing")
    ap.add_argument("--no-models", action="store_true",
                    help="skip the gradient-domain and one-bit ADMM steps and the "
                         "fixed-accuracy Tucker prox")
    ap.add_argument("--slice-kernels", action="store_true",
                    help="take --warmup eager steps of the workload, time every kernel of one "
                         "slice pass on the iterate, print them and exit (a small, short case "
                         "for kernel profilers)")
    ap.add_argument("--learned-iters", type=int, default=100)
    ap.add_argument("--batch-steps", type=int, default=8)
    return ap.parse_args()


def max_over_ranks(dist, value, device):
    """MAX of a float over all ranks: a job's time is its slowest rank's."""
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput of `world` replicas that each processed
    `units_per_rank` units, timed by the slowest rank (weak scaling)."""
    return units_per_rank * world / seconds


def replica_seed(base_seed, rank):
    """Each rank recovers its own replica of the workload."""
    return base_seed + rank


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------ CPU oracle leg
def oracle_steps(workload, budget_s, max_steps, warmup=0, engine="rsvd"):
    """Time the FP64 oracle's ADMM iteration on the workload (host cores);
    engine "rsvd" is the randomized prox of the GPU path, "full" the
    deterministic GNHTSVT (a full SVD of every transformed slice)."""
    import numpy as np
    from oracle import admm
    from paper_2506_09594_gb300 import synth
    w = synth.WORKLOADS[workload]
    _, M, mask, _ = synth.make_problem(w)
    p = admm.Params(lam=admm.default_lambda(w.n1, w.n2, w.tdims), engine=engine, l=w.l, q=w.q,
                    seed=w.seed, noise=admm.NOISE_NONE if w.noise_model == "none"
                    else admm.NOISE_L1)
    st = admm.init_state(M.shape, p.mu0)
    for _ in range(warmup):
        st, _ = admm.step(st, M, mask, w.tdims, p)
    done, t0 = 0, time.perf_counter()
    while done < max_steps:
        st, _ = admm.step(st, M, mask, w.tdims, p)
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    return done, el


def cpu_child(args):
    done, el = oracle_steps(args.workload, args.cpu_seconds, 1000, engine=args.cpu_engine)
    print(json.dumps({"steps": done, "seconds": el}))


def cpu_baseline(workload, seconds, cores=None, engine="rsvd"):
    """Run the oracle in a child process with `cores` BLAS threads (default:
    every host core)."""
    from paper_2506_09594_gb300 import synth
    w = synth.WORKLOADS[workload]
    cores = cores or os.cpu_count() or 1
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-child", "--workload",
                          workload, "--cpu-seconds", str(seconds), "--cpu-engine", engine],
                         capture_output=True, text=True, env=env, timeout=600)
    line = [l for l in out.stdout.splitlines() if l.startswith("{")]
    if out.returncode != 0 or not line:
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": "failed: " + out.stderr[-300:]}
    r = json.loads(line[-1])
    what = ("randomized engine l=%d q=%d" % (w.l, w.q) if engine == "rsvd"
            else "deterministic engine: full SVD of every transformed slice")
    return {"value": r["steps"] / r["seconds"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d full ADMM iterations of %s (numpy float64, %s), %.1f s"
                      % (r["steps"], workload, what, r["seconds"])}


# ------------------------------------------------------------ clock sampler
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- our arm
def tube_forward_bytes(N, esz):
    # reads M, L, E, Y, G, Lambda (esz each) and the 1-byte mask; writes L, E, Y, Abar
    return N * (6 * esz + 1 + 4 * esz)


def tube_inverse_bytes(N, esz):
    # reads Gbar, L, G, Lambda; writes G, Lambda
    return N * 6 * esz


# DRAM traffic of one tube_fused_kernel launch on the bench workload, from the
# ncu capture summarised in profiles/tube_fused_kernel_tubal200x400_r10.md,
# valid only while the kernel source is the one that was profiled.
TUBE_FUSED_TRAFFIC = {"workload": "tubal200x400_r10", "src_sha256_prefix": "0b78584641edc851",
                      "bytes": 467.097088e6 + 329.501952e6}


def profiled_traffic(workload):
    import hashlib
    path = os.path.join(ROOT, "paper_2506_09594_gb300", "csrc", "tube_kernels.cu")
    try:
        sha = hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    t = TUBE_FUSED_TRAFFIC
    return t["bytes"] if (sha == t["src_sha256_prefix"] and workload == t["workload"]) else None


def tube_fused_bytes(N, esz):
    # the fused tube pass's algorithmic bytes: reads M, L, E, Y, Lambda, Gbar
    # (esz each) and the 1-byte mask, writes L, E, Y, Lambda, Abar
    return N * (11 * esz + 1)


def tube_fused_bytes_g(N, esz):
    # the same plus the G stream the kernel also carries: G^t read and
    # G^{t+1} written, for ||G^{t+1} - G^t||_inf of the stop test
    return N * (13 * esz + 1)


def kernel_rooflines(kernels, w, esz, hbm_peak, tflops_peak):
    """Per-kernel rooflines of one slice pass from its CUDA-event times
    (tr_profile_slice_pass): algorithmic bytes of each kernel (what it must
    read and write: the transformed slice stack for the products, the panels
    for the QRs and the SVD core, the panels and Gbar for the rebuild) over
    its device time, against the measured HBM copy peak; the tensor-core
    products also give their MMA rate against the measured BF16 peak."""
    n, n1, n2, l = w.nslices, w.n1, w.n2, min(w.l, w.n1, w.n2)
    A = n * n1 * n2 * esz
    out, last_rows = [], n1
    for name, ms in kernels:
        flops = None
        if name == "sketch":
            b = n * n2 * l * esz
        elif name.startswith("product A*X"):
            b = A + n * (n2 + n1) * l * esz
            last_rows = n1
            flops = 2.0 * n * n1 * n2 * l * (3 if "split" in name else 1)
        elif name.startswith("product A^T*Q"):
            b = A + n * (n1 + n2) * l * esz
            last_rows = n2
            flops = 2.0 * n * n1 * n2 * l * (3 if "split" in name else 1)
        elif name == "qr":
            b = 2 * n * last_rows * l * esz
        elif name == "svd_core":
            b = n * (2 * n1 + n2) * l * esz
        elif name == "rank_update":
            b = n * (n1 + n2) * l * esz + A
        elif name == "svd_core + rank_update":   # the core writing Gbar itself
            b = n * (n1 + n2) * l * esz + A
        else:
            b = None
        gbs = b / (ms * 1e-3) / 1e9 if (b and ms > 0) else None
        e = {"kernel": name, "ms": ms, "bound": "hbm", "algorithmic_bytes": b,
             "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
             "frac": gbs / hbm_peak if gbs else None}
        if flops and "tcgen05" in name and ms > 0:
            e["tensor_tflops"] = flops / (ms * 1e-3) / 1e12
            e["tensor_frac"] = e["tensor_tflops"] / tflops_peak
        out.append(e)
    return out


def oracle_parity(w, M, mask, states, tol, steps=2, noise_model=None):
    """The FP64 oracle's `steps` ADMM steps from the GPU's state s0 against
    the GPU's state after the same steps (an eager step, then replays of the
    timed graph): relative Frobenius error and largest elementwise error
    (over the largest |value|) of L, E, Y, Lambda and G."""
    import numpy as np
    from oracle import admm
    s0, s2 = states
    nm = noise_model or w.noise_model
    p = admm.Params(lam=admm.default_lambda(w.n1, w.n2, w.tdims), engine="rsvd", l=w.l, q=w.q,
                    seed=w.seed, noise=admm.NOISE_NONE if nm == "none" else admm.NOISE_L1)
    f64 = lambda a: np.asarray(a, dtype=np.float64)
    st = admm.State(L=f64(s0["L"]), E=f64(s0["E"]), Y=f64(s0["Y"]), Lam=f64(s0["Lam"]),
                    G=f64(s0["G"]), mu=float(s0["mu"]), t=int(s0["t"]))
    Mq = f64(np.asarray(M, dtype=np.float32) if w.dtype == "f32" else M)
    t0 = time.perf_counter()
    for _ in range(steps):
        st, _ = admm.step(st, Mq, mask, w.tdims, p)
    el = time.perf_counter() - t0
    out = {"steps": steps, "from_iteration": int(s0["t"]), "tol": tol, "oracle_s": el}
    ok = True
    for name in ("L", "E", "Y", "Lam", "G"):
        want = getattr(st, name)
        got = f64(s2[name])
        nw = float(np.linalg.norm(want))
        rel = float(np.linalg.norm(got - want) / nw) if nw > 0 else float(np.linalg.norm(got))
        mx = float(np.abs(want).max())
        mabs = float(np.abs(got - want).max() / mx) if mx > 0 else float(np.abs(got).max())
        out[name] = {"rel_F": rel, "max_abs_over_max": mabs}
        if name == "Lam" and steps == 1:
            # Lambda+ = Lambda + mu (L - G): after one step from the same
            # state its error is mu times that of L - G, however small
            # Lambda itself is; that derived bound is the test
            dL = float(np.linalg.norm(f64(s2["L"]) - st.L))
            dG = float(np.linalg.norm(f64(s2["G"]) - st.G))
            bound = float(s0["mu"]) * (dL + dG) * 1.001 + tol * nw
            err = float(np.linalg.norm(got - want))
            out[name]["bound_mu_dL_dG"] = bound
            ok = ok and err <= bound
        else:
            ok = ok and rel <= tol and mabs <= tol
    out["pass"] = ok
    return out


PREC = {"fp32": 0, "bf16": 2, "bf16x3": 3}


def make_handle(tr, torch, w, Md, maskd, stream, rank, prec):
    rank_k = int(w.rank) if w.rank != "powerlaw" else 10
    return tr.Handle(Md, maskd, w.dims, stream=stream.cuda_stream, rank=rank_k,
                     oversample=w.l - rank_k, power_iters=w.q, seed=replica_seed(w.seed, rank), prec=prec,
                     noise=tr.TR_NOISE_NONE if w.noise_model == "none" else tr.TR_NOISE_L1)


def time_form(tr, torch, dist, w, Md, maskd, X_dev, stream, rank, world, prec, K, W, clocks=None,
              chosen=False):
    """Warm up W steps, then time K steps of one form; returns its measurements.

    The plain form runs eager launches with per-phase events in the timed
    region.  The chosen form replays one CUDA graph per step with the
    autotuned tube tile; its phases come from a profiled eager window of the
    same kernels right after the timed region."""
    with torch.cuda.stream(stream):
        h = make_handle(tr, torch, w, Md, maskd, stream, rank, prec)
    tune = None
    warm = W
    if chosen:
        h.step()                  # first warm-up step, then tune on L(M)
        warm -= 1
        tune = h.autotune(5)      # leaves the iterate as it was
        h.graph_mode(True)
    for _ in range(warm):
        h.step()
    if not chosen:
        h.profile_enable(K)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    if clocks is not None:
        clocks.start()
        time.sleep(0.3)
    launches0 = h.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(K):
        h.step()
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = h.kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop() if clocks is not None else None
    if world > 1:
        ms = max_over_ranks(dist, ms, "cuda")
        dist.barrier()
    L = h.get_state()["L"]
    rec = float(torch.linalg.norm((L - X_dev).double()) / torch.linalg.norm(X_dev.double()))
    parity = None
    kernels = None
    if chosen:
        # oracle parity of the timed configuration: the state s0 here, then
        # one eager step and one replay of the timed graph (the fused tube
        # pass completes the first step inside the second); the FP64 oracle
        # takes the same two steps from s0 in the CPU leg
        s0 = h.get_state()
        h.step()
        h.step()
        s2 = h.get_state()
        to_host = lambda d: {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in d.items()}
        parity = (to_host(s0), to_host(s2))
        # per-kernel device times of one slice pass on this iterate's
        # transformed tensor Abar = L(L + Lambda / mu), tau = 1 / mu
        X = (s2["L"] + s2["Lam"] / s2["mu"]).contiguous()
        torch.cuda.synchronize()
        Ab = h.transform_forward(X)
        kernels = h.profile_slice_pass(Ab, 1.0 / s2["mu"], s2["t"], reps=5)
        torch.cuda.synchronize()
        del Ab, X, s0, s2
    if chosen:
        KP = max(3, min(K, 10))
        h.profile_enable(KP)
        for _ in range(KP):
            h.step()
    phases = h.profile_read()
    return h, {"ms": ms, "phases": phases, "launches": launches, "clocks": clk,
               "recovery_rel_err": rec, "L": L, "tube_tile": tune, "parity": parity,
               "kernels": kernels}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2506_09594_gb300 import synth, tr

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    tr.load()
    w = synth.WORKLOADS[args.workload]
    dt = torch.float64 if w.dtype == "f64" else torch.float32
    esz = 8 if w.dtype == "f64" else 4
    X, M, mask, _ = synth.make_problem(w, seed=replica_seed(w.seed, rank))
    M_host = torch.from_numpy(M).to(dt).pin_memory()
    mask_host = torch.from_numpy(mask).pin_memory()
    Md = M_host.to("cuda")
    maskd = mask_host.to("cuda")
    X_dev = torch.from_numpy(X).to("cuda", dt)
    stream = torch.cuda.Stream()
    K, W = args.steps, args.warmup
    chosen = PREC[args.prec] if w.dtype != "f64" else 0

    # plain form: FP32 SIMT products (the speedup denominator)
    hp, plain = time_form(tr, torch, dist, w, Md, maskd, X_dev, stream, rank, world, 0, K, W)
    hp.close()
    # chosen form (tensor-core products), timed with the clock sampler running
    clocks = ClockSampler(local)
    h, ch = time_form(tr, torch, dist, w, Md, maskd, X_dev, stream, rank, world, chosen, K, W,
                      clocks, chosen=True)
    agree = float(torch.linalg.norm((ch["L"] - plain["L"]).double())
                  / torch.linalg.norm(plain["L"].double()).clamp_min(1e-300))
    ms, phases = ch["ms"], ch["phases"]
    # the single-pass BF16 form (stated bound 1e-3), timed the same way, as a
    # second arm beside the headline form
    alt = None
    if chosen == 3:
        ha, alt = time_form(tr, torch, dist, w, Md, maskd, X_dev, stream, rank, world, 2, K, W,
                            chosen=True)
        ha.close()
        torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers: every step copies the
    # problem's inputs (observed values, mask) from pinned host memory and
    # reads the step's result (its residual maxima, tr_read_residuals) back
    # into pinned host memory.  The copy of step k+1's inputs runs on a copy
    # stream into the second of two device buffers while step k computes
    # (tr_set_observed swaps the buffers; the handle keeps one captured step
    # graph per buffer pair, both captured by two untimed steps).
    KE = max(3, min(K, 20))
    h.graph_mode(True)
    bufs = [(Md, maskd), (torch.empty_like(Md), torch.empty_like(maskd))]
    copy_stream = torch.cuda.Stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    used = [torch.cuda.Event(), torch.cuda.Event()]
    res_host = torch.zeros(10 * KE, dtype=torch.float64).pin_memory()

    def upload(k):
        dm, dk = bufs[k % 2]
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(used[k % 2])      # step k-2 read this buffer
            dm.copy_(M_host, non_blocking=True)
            dk.copy_(mask_host, non_blocking=True)
            copied[k % 2].record(copy_stream)

    def run(steps):
        upload(0)
        for k in range(steps):
            stream.wait_event(copied[k % 2])
            h.set_observed(*bufs[k % 2])
            if k + 1 < steps:
                upload(k + 1)
            h.step()
            h.read_residuals(res_host[10 * k:10 * k + 10])
            used[k % 2].record(stream)

    L_host = torch.empty(M_host.shape, dtype=dt).pin_memory()
    run(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run(KE)
    # the recovery's result: L back to pinned host memory once, after the
    # last step (its cost is spread over the KE steps in d2h_bytes_per_step)
    L_host.copy_(h.get_L(), non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if not bool(torch.isfinite(res_host).all()):
        raise RuntimeError("non-finite residuals in the end-to-end steps")
    h.set_observed(Md, maskd)
    if world > 1:
        e2e_s = max_over_ranks(dist, e2e_s, "cuda")

    N = w.numel
    n = w.nslices
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    # steps without info run the fused tube kernel (inverse of the previous
    # step + forward of this one) and no separate inverse kernel
    fwd_ms = phases["tube_forward"]
    fwd_gbs = tube_fused_bytes(N, esz) / (fwd_ms * 1e-3) / 1e9 if fwd_ms > 0 else None
    fwd_gbs_g = tube_fused_bytes_g(N, esz) / (fwd_ms * 1e-3) / 1e9 if fwd_ms > 0 else None
    step_bytes = tube_fused_bytes(N, esz) + 2 * N * esz
    slice_ms = phases["slice_pass"]
    slice_gbs = 2 * N * esz / (slice_ms * 1e-3) / 1e9 if slice_ms > 0 else None
    kern_roof = kernel_rooflines(ch["kernels"] or [], w, esz, hbm_peak,
                                 peaks.get("bf16_tflops", 1899.5))
    value = job_rate(K, world, ms * 1e-3)
    plain_value = job_rate(K, world, plain["ms"] * 1e-3)
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": world,
            "steps": K,
            "warmup": W,
            "ms_per_step": ms / K,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": w.dtype,
            "data": "synthetic (seeded; tensors shaped like the paper's workloads)",
            "impl": "ours",
            "config": {
                "workload": args.workload,
                "dims": list(w.dims),
                "slices": n,
                "rank": w.rank,
                "sketch_width": w.l,
                "power_iters": w.q,
                "sampling_ratio": w.sr,
                "form": {0: "fp32 simt", 2: "bf16 tcgen05 (split-bf16 refinement)",
                         3: "split-bf16 tcgen05"}[chosen] + ", graph replay, autotuned tube tile "
                         "and slice split",
                "tube_tile": ch["tube_tile"][0] if ch["tube_tile"] else None,
                "slice_groups": ch["tube_tile"][1] if ch["tube_tile"] else None,
                "parallelism": "replicas" if world > 1 else "single",
                "l2": "state 7 x %.0f MB >> 129 MB L2: no flush needed" % (N * esz / 1e6),
            },
            "plain": {"value": plain_value, "ms_per_step": plain["ms"] / K,
                      "form": "fp32 simt", "phases_ms": plain["phases"],
                      "recovery_rel_err": plain["recovery_rel_err"]},
            "speedup_vs_plain": value / plain_value,
            "bf16_form": None if alt is None else {
                "value": job_rate(K, world, alt["ms"] * 1e-3), "ms_per_step": alt["ms"] / K,
                "form": "bf16 tcgen05 (split-bf16 refinement of the last two products), graph "
                        "replay", "stated_bound": 1e-3,
                "speedup_vs_plain": plain["ms"] / alt["ms"],
                "recovery_rel_err": alt["recovery_rel_err"]},
            "recovery_rel_err": ch["recovery_rel_err"],
            "chosen_vs_plain_L_rel_diff": agree,
            "gpu_launches": int(ch["launches"]),
            "roofline": {
                "kernel": "tube_fused_kernel",
                "bound": "hbm",
                "achieved": fwd_gbs,
                "peak": hbm_peak,
                "unit": "GB/s",
                "frac": (fwd_gbs / hbm_peak) if fwd_gbs else None,
                "traffic": profiled_traffic(args.workload),
                "peak_source": peak_src,
                "algorithmic_bytes": tube_fused_bytes(N, esz),
                "bytes_per_element": "45: reads M, L, E, Y, Lambda, Gbar (4 B each) and the "
                                     "mask (1 B), writes L, E, Y, Lambda, Abar",
                "with_g_stream": {"bytes_per_element": 53, "achieved": fwd_gbs_g,
                                  "frac": (fwd_gbs_g / hbm_peak) if fwd_gbs_g else None,
                                  "why": "G read and written: ||G^{t+1} - G^t||_inf of the "
                                         "stop test (Eq. convercon)"},
            },
            "roofline_slice_pass": {
                "bound": "hbm", "ms": slice_ms, "algorithmic_bytes": 2 * N * esz,
                "bytes": "Abar read once, Gbar written once", "achieved": slice_gbs,
                "peak": hbm_peak, "unit": "GB/s",
                "frac": (slice_gbs / hbm_peak) if slice_gbs else None,
            },
            "roofline_kernels": kern_roof,
            "phases_ms": {"tube_fused": fwd_ms, "slice_pass": phases["slice_pass"]},
            "step_hbm_fraction": (step_bytes / (ms / K * 1e-3) / 1e9) / hbm_peak,
            "e2e": {"value": job_rate(KE, world, e2e_s), "unit": UNIT,
                    "h2d_bytes_per_step": int(N * esz + N),
                    "d2h_bytes_per_step": int(8 * 10 + N * esz / KE),
                    "form": "graph replay per buffer pair, uploads overlapped on a copy stream, "
                            "residuals read back every step, L read back once after the last "
                            "step (%d steps)" % KE},
            "clocks": ch["clocks"],
        }
    h.close()
    del Md, maskd, X_dev
    torch.cuda.empty_cache()
    if rank == 0:
        if not args.no_learned and world == 1:
            line["learned"] = learned_ab(tr, torch, args.learned_iters, chosen)
            torch.cuda.empty_cache()
        if not args.no_batch and world == 1:
            line["batch"] = batch_bench(tr, torch, args.batch_steps, chosen)
            torch.cuda.empty_cache()
        if not args.no_precision and world == 1:
            line["precision"] = precision_forms(tr, torch, 20)
            torch.cuda.empty_cache()
        if not args.no_tucker and world == 1:
            line["tucker"] = tucker_section(tr, torch)
            torch.cuda.empty_cache()
        if not args.no_models and world == 1:
            line["models"] = models_section(tr, torch, 20)
            torch.cuda.empty_cache()
        if not args.no_small and world == 1:
            line["small"] = small_section(tr, torch, K, W, args.no_cpu_baseline)
            torch.cuda.empty_cache()
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_seconds)
            # the rest of the CPU plan: the same oracle on one core, and the
            # deterministic (full-SVD) oracle, on bounded samples
            line["cpu_baseline"]["one_core"] = cpu_baseline(args.workload,
                                                            args.cpu_seconds / 2, cores=1)
            line["cpu_baseline"]["deterministic"] = cpu_baseline(args.workload,
                                                                 args.cpu_seconds / 2,
                                                                 engine="full")
            # the timed forms against the FP64 oracle on the same two steps
            line["oracle_parity"] = oracle_parity(w, M, mask, ch["parity"], 1e-4)
            if alt is not None:
                line["bf16_form"]["oracle_parity"] = oracle_parity(w, M, mask, alt["parity"],
                                                                   1e-3)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def small_section(tr, torch, K, W, no_cpu):
    """The small workload (64x64x16 FP64, tubal rank 5, 50% observed,
    noise-free, l = 15, q = 1): the graph-replayed FP64 form timed like the
    headline, its oracle parity (two steps from the state after the timed
    steps, stated bound 1e-10 for FP64), and the oracle's own rate on all
    cores and on one, randomized and deterministic (these runs are short)."""
    import numpy as np
    from paper_2506_09594_gb300 import synth
    w = synth.WORKLOADS["tubal64_r5"]
    X, M, mask, _ = synth.make_problem(w)
    Md = torch.from_numpy(M).to("cuda", torch.float64)
    maskd = torch.from_numpy(mask).cuda()
    Xd = torch.from_numpy(X).to("cuda", torch.float64)
    stream = torch.cuda.Stream()
    h, r = time_form(tr, torch, None, w, Md, maskd, Xd, stream, 0, 1, 0, K, W, chosen=True)
    h.close()
    out = {"workload": w.name, "dims": list(w.dims), "dtype": "f64",
           "value": K / (r["ms"] * 1e-3), "unit": UNIT, "ms_per_step": r["ms"] / K,
           "form": "fp64 simt, graph replay, autotuned tube tile and slice split",
           "recovery_rel_err": r["recovery_rel_err"], "gpu_launches": int(r["launches"])}
    if not no_cpu:
        out["oracle_parity"] = oracle_parity(w, M, mask, r["parity"], 1e-10)
        out["cpu_baseline"] = cpu_baseline(w.name, 5.0)
        out["cpu_baseline"]["one_core"] = cpu_baseline(w.name, 5.0, cores=1)
        out["cpu_baseline"]["deterministic"] = cpu_baseline(w.name, 5.0, engine="full")
    return out


def learned_ab(tr, torch, iters, prec):
    """The learned widths against the method without them, on the
    512x512x32x16 power-law workload, at equal recovery error.  The plain
    method is the adaptive engine (Alg. 3 per slice, eps 0.01, block 10, cap
    70), which is also the learned engine's judge and fallback; it runs
    `iters` iterations.  The learned engine, in FP32 (the plain method's
    precision) and in the chosen tensor-core form, then runs until its
    recovery error is within 1e-4 of the plain method's (at most `iters` + 40
    iterations).  The fixed-width engine (l = 74, FP32) runs `iters`
    iterations for context.  Times are the summed device time of the steps;
    fallback_slices_total counts the slices Alg. 3's judge rejected."""
    from paper_2506_09594_gb300 import synth
    w = synth.WORKLOADS["tubal512x512_powerlaw"]
    X, M, mask, ranks = synth.make_problem(w)
    Md = torch.from_numpy(M).float().cuda()
    maskd = torch.from_numpy(mask).cuda()
    Xd = torch.from_numpy(X).float().cuda()
    Xn = float(torch.linalg.norm(Xd.double()))
    del X, M, mask
    out = {"workload": w.name, "dims": list(w.dims), "sampling_ratio": w.sr,
           "slice_ranks": "power law on [2, 64], mean %.1f" % float(ranks.mean()),
           "iters_plain": iters, "l_max": 74, "schedule": "mu0 1e-3, growth 1.1",
           "criterion": "recovery rel-err within +1e-4 of the plain (adaptive) method after "
                        "iters_plain"}
    stream = torch.cuda.Stream()
    forms = {0: "fp32 simt", 2: "bf16 tcgen05", 3: "split-bf16 tcgen05"}

    def err_of(h):
        L = h.get_L()
        return float(torch.linalg.norm((L - Xd).double())) / Xn

    target = None
    arms = (("adaptive", tr.TR_LR_ADAPTIVE, 0), ("learned_fp32", tr.TR_LR_LEARNED, 0),
            ("learned_%s" % {0: "fp32", 2: "bf16", 3: "bf16x3"}[prec], tr.TR_LR_LEARNED, prec),
            ("fixed_width", tr.TR_LR_RSVD, 0))
    seen = set()
    for name, eng, pr in arms:
        if name in seen:
            continue
        seen.add(name)
        kw = dict(engine=eng, rank=64, oversample=6 if eng == tr.TR_LR_ADAPTIVE else 10,
                  noise=tr.TR_NOISE_NONE, seed=w.seed, tol=0.0, max_iter=iters, prec=pr,
                  adapt_eps=0.01, adapt_block=10, stream=stream.cuda_stream)
        if eng == tr.TR_LR_LEARNED:
            kw["model_path"] = tr.DEFAULT_MODEL.encode()
        h = tr.Handle(Md, maskd, w.dims, **kw)
        ms, fb, it, err = 0.0, 0, 0, None
        chase = eng == tr.TR_LR_LEARNED
        limit = iters + 40 if chase else iters
        while it < limit:
            info = h.step(info=True)
            ms += info["ms"]
            fb += info["fallback_slices"]
            it += 1
            if chase and it >= iters - 10 and it % 2 == 0:
                err = err_of(h)
                if err <= target + 1e-4:
                    break
        if err is None or not chase:
            err = err_of(h)
        if name == "adaptive":
            target = err
        widths = h.slice_widths()
        out[name] = {"iterations": it, "device_ms": ms, "iters_per_s": it / (ms * 1e-3),
                     "recovery_rel_err": err, "reached_target": err <= target + 1e-4,
                     "mean_width_last": float(widths.mean()), "fallback_slices_total": fb,
                     "slice_passes": it * w.nslices, "kernel_launches": h.kernel_launches(),
                     "form": {tr.TR_LR_ADAPTIVE: "Alg. 3 per slice, eps 0.01, block 10, cap 70",
                              tr.TR_LR_LEARNED: "learned widths, Alg. 3 judge and fallback",
                              tr.TR_LR_RSVD: "fixed width l = 74"}[eng] + ", " + forms[pr]}
        h.close()
    base_ms = out["adaptive"]["device_ms"]
    out["speedup_at_equal_error"] = {k: (base_ms / out[k]["device_ms"] if out[k]["reached_target"]
                                         else None)
                                     for k in out if k.startswith("learned_")}
    out["speedup_per_iteration"] = {k: out[k]["iters_per_s"] / out["adaptive"]["iters_per_s"]
                                    for k in out if k.startswith("learned_") or k == "fixed_width"}
    return out


def tucker_section(tr, torch, reps=20):
    """The paper's own randomized GNHTSVT (shared Tucker factors of the two
    spatial modes, Alg. 1 + Alg. 4 randomized branch) beside the per-slice
    randomized prox, on a 200x200x20x20 FP32 transformed stack whose slices
    share column and row spaces of dimension 10 (plus 1e-3 noise): device ms
    per prox (CUDA events; the Tucker call's workspace comes from the
    stream-ordered allocator inside the timed region) and the relative
    difference of the two results."""
    dims, n, n1, n2, sdim = (200, 200, 20, 20), 400, 200, 200, 10
    g = torch.Generator(device="cuda").manual_seed(7)
    P = torch.linalg.qr(torch.randn(n1, sdim, device="cuda", generator=g))[0]
    Q = torch.linalg.qr(torch.randn(n2, sdim, device="cuda", generator=g))[0]
    S = 3.0 * torch.randn(n, sdim, sdim, device="cuda", generator=g)
    Ab = (P @ S @ Q.T + 1e-3 * torch.randn(n, n1, n2, device="cuda", generator=g)).float()
    # blocks at least the shared dimension (with a flat signal spectrum
    # (A A^T) A G is nearly parallel to A G, so smaller blocks miss part of
    # the shared spaces) and one Krylov step (the sketch of an unfolding
    # with n n2 columns gathers the noise of every slice)
    r, b, q = (16, 16), (16, 16), (1, 1)
    G1 = torch.randn(b[0], n * n2, device="cuda", generator=g)   # column-major (n n2) x b1
    G2 = torch.randn(b[1], n * r[0], device="cuda", generator=g)
    M = torch.zeros_like(Ab)
    mask = torch.ones(Ab.shape, dtype=torch.uint8, device="cuda")
    h = tr.Handle(M, mask, dims, phi=tr.TR_PEN_L1, rank=r[0], oversample=0, power_iters=1)
    tau = 1.0
    out_t, out_r = torch.empty_like(Ab), torch.empty_like(Ab)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_t = timed(lambda: h.slice_prox_tucker(Ab, tau, r, b, q, G1, G2, out=out_t))
    ms_r = timed(lambda: h.slice_prox(Ab, tau, 0, out=out_r))
    diff = float(torch.linalg.norm((out_t - out_r).double())
                 / torch.linalg.norm(out_r.double()).clamp_min(1e-300))
    h.close()
    return {"workload": "200x200x20x20 FP32 transformed stack, shared column/row spaces of "
                        "dimension 10, noise 1e-3, l1 shrink tau 1",
            "tucker": {"ranks": list(r), "blocks": list(b), "krylov": list(q),
                       "ms_per_prox": ms_t},
            "per_slice_rsvd": {"l": r[0], "q": 1, "ms_per_prox": ms_r},
            "rel_diff_tucker_vs_per_slice": diff}


def models_section(tr, torch, K):
    """The two other models of the paper on the headline shape, 200x200x20x20
    FP32 (400 slices), Gamma = {1, 2}, per-slice randomized prox with l = 20
    and q = 1: device ms per ADMM step (CUDA events over K steps after 3
    warm-up steps).  The gradient-domain prior (Alg. 5 with Gamma) runs on the
    headline observed data; the one-bit model (Alg. 6) on 2N dithered signs
    of its ground truth (theta = 1.2 max |X*|)."""
    import numpy as np

    from paper_2506_09594_gb300 import synth
    w = synth.WORKLOADS[WORKLOAD]
    X, M, mask, _ = synth.make_problem(w)
    out = {"workload": w.name, "modes": [1, 2],
           "sketch_width": 20, "power_iters": 1, "steps": K}

    def timed(step):
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            step()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K

    Md = torch.from_numpy(M).float().cuda()
    maskd = torch.from_numpy(mask).cuda()
    c = tr.Ctv(Md, maskd, w.dims, modes=[1, 2], rank=10, oversample=10, power_iters=1,
               stream=torch.cuda.current_stream().cuda_stream)
    ms = timed(c.step)
    out["ctv"] = {"ms_per_step": ms, "iters_per_s": 1e3 / ms}
    c.close()
    del Md, maskd
    torch.cuda.empty_cache()
    rng = np.random.default_rng(11)
    theta = 1.2 * float(np.abs(X).max())
    s, q = synth.one_bit_observations(X, 2 * X.size, theta, 0.0, rng)
    ob = tr.OneBit(w.dims, torch.from_numpy(s).cuda(), torch.from_numpy(q.astype(np.int8)).cuda(),
                   modes=[1, 2], rank=10, oversample=10, power_iters=1, theta=theta,
                   alpha=float(np.abs(X).max()), stream=torch.cuda.current_stream().cuda_stream)
    ms = timed(ob.step)
    out["onebit"] = {"ms_per_step": ms, "iters_per_s": 1e3 / ms, "samples": int(len(s))}
    ob.close()
    # the fixed-accuracy shared-Tucker prox (Alg. AD-RSTHOSVD-BLBP + Alg. 4) on
    # a 200x200x20x20 FP32 transformed stack sharing spaces of dimension 10
    g = torch.Generator(device="cuda").manual_seed(7)
    n, n1, n2, sdim = 400, 200, 200, 10
    P = torch.linalg.qr(torch.randn(n1, sdim, device="cuda", generator=g))[0]
    Q = torch.linalg.qr(torch.randn(n2, sdim, device="cuda", generator=g))[0]
    Ab = torch.einsum("ia,jab,kb->jik", P, 3.0 * torch.randn(n, sdim, sdim, device="cuda",
                                                             generator=g), Q).contiguous()
    Ab += 1e-3 * torch.randn(Ab.shape, device="cuda", generator=g)
    res = {}
    ms = timed(lambda: res.__setitem__("r", tr.slice_prox_ad_tucker(Ab, 1.0, 1e-2, 10,
                                                                    delta_rel=1e-5,
                                                                    phi=tr.TR_PEN_L1)[1]))
    out["ad_tucker"] = {"ms_per_prox": ms, "eps": 1e-2, "block": 10, "ranks": list(res["r"])}
    return out


def precision_forms(tr, torch, K):
    """The three operand forms on the 1024x1024x64 workload (rank 32, 20%
    observed, l = 48): device ms per step (graph replay with the autotuned
    tube tile and slice split, K steps after 5 warm-up steps), the relative Frobenius difference of L from the plain
    FP32 form after the same steps, and each form's parity with the FP64
    oracle for one step from its state after them (tolerance 1e-4 for the
    FP32 and split-BF16 forms, 1e-3 for the BF16 form)."""
    from paper_2506_09594_gb300 import synth
    w = synth.WORKLOADS["tubal1024x64_r32"]
    X, M, mask, _ = synth.make_problem(w)
    Md = torch.from_numpy(M).float().cuda()
    maskd = torch.from_numpy(mask).cuda()
    Xd = torch.from_numpy(X).float().cuda()
    del X
    stream = torch.cuda.Stream()
    out = {"workload": w.name, "dims": list(w.dims), "rank": w.rank, "sketch_width": w.l,
           "sampling_ratio": w.sr, "steps": K, "schedule": "mu0 0.05, growth 1.1"}
    Ls = {}
    for name, pr in (("fp32", 0), ("bf16x3", 3), ("bf16", 2)):
        # mu0 0.05: after the warm-up steps tau = 1/mu has fallen below the
        # observed slices' leading singular values, so the prox keeps ranks
        h = tr.Handle(Md, maskd, w.dims, rank=w.l, oversample=0, power_iters=w.q, seed=w.seed,
                      prec=pr, noise=tr.TR_NOISE_NONE, mu0=0.05, stream=stream.cuda_stream)
        # as the headline form: tube tile and slice split autotuned after the
        # first step (the tuner leaves the iterate as it was)
        h.step()
        tune = h.autotune(5)
        h.graph_mode(True)
        for _ in range(4):
            h.step()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(K):
            h.step()
        ev1.record(stream)
        torch.cuda.synchronize()
        # phases of a few eager steps (tube pass, slice pass)
        h.profile_enable(3)
        for _ in range(3):
            h.step()
        ph = h.profile_read()
        L = h.get_L()
        Ls[name] = L
        out[name] = {"ms_per_step": ev0.elapsed_time(ev1) / K,
                     "tube_tile": tune[0], "slice_groups": tune[1],
                     "phases_ms": {"tube_forward": ph["tube_forward"],
                                   "slice_pass": ph["slice_pass"]},
                     "recovery_rel_err": float(torch.linalg.norm((L - Xd).double())
                                               / torch.linalg.norm(Xd.double()))}
        # one more step of this form against the oracle's step from the same state
        to_host = lambda d: {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in d.items()}
        s0 = to_host(h.get_state())
        h.step()
        s1 = to_host(h.get_state())
        h.close()
        out[name]["oracle_parity"] = oracle_parity(w, M, mask, (s0, s1),
                                                   1e-3 if name == "bf16" else 1e-4, steps=1,
                                                   noise_model="none")
        del s0, s1
    base = Ls["fp32"].double()
    for name in ("bf16x3", "bf16"):
        out[name]["L_rel_diff_vs_fp32"] = float(torch.linalg.norm(Ls[name].double() - base)
                                                / torch.linalg.norm(base).clamp_min(1e-300))
        out[name]["speedup_vs_fp32"] = out["fp32"]["ms_per_step"] / out[name]["ms_per_step"]
    return out


def batch_problems(torch, tr, count, seed):
    """64 problems of uneven shapes, generated on the device: transform-domain
    slices A_j B_j^T / sqrt(r) (N(0,1) factors), mapped back with the
    problem's own inverse transform, Bernoulli(SR) mask."""
    import numpy as np
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(count):
        n1, n2 = int(rng.integers(128, 769)), int(rng.integers(128, 769))
        n3 = int(rng.integers(8, 65))
        dims = (n1, n2, n3) if rng.random() < 0.5 else (n1, n2, n3, int(rng.integers(4, 17)))
        specs.append({"dims": dims, "rank": int(rng.integers(4, 41)),
                      "sr": float(rng.uniform(0.10, 0.50))})
    return specs


def batch_bench(tr, torch, K, prec):
    specs = batch_problems(torch, tr, 64, 2000)
    g = torch.Generator(device="cuda")
    g.manual_seed(2000)
    probs, prms, elems = [], [], 0
    for i, sp in enumerate(specs):
        dims = sp["dims"]
        n = 1
        for d in dims[2:]:
            n *= d
        n1, n2, r = dims[0], dims[1], sp["rank"]
        A = torch.randn((n, n1, r), generator=g, device="cuda")
        B = torch.randn((n, n2, r), generator=g, device="cuda")
        Xbar = torch.bmm(A, B.transpose(1, 2)) / (r ** 0.5)
        del A, B
        mask = (torch.rand((n, n1, n2), generator=g, device="cuda") < sp["sr"]).to(torch.uint8)
        probs.append([Xbar, mask, dims])
        prms.append(tr.default_params(rank=r, oversample=10, seed=2000 + i, prec=prec,
                                      noise=tr.TR_NOISE_NONE))
        elems += n * n1 * n2
    out = {"problems": len(specs), "elements": elems,
           "shapes": "n1, n2 ~ U{128..768}, n3 ~ U{8..64}, order 4 w.p. 1/2 with n4 ~ U{4..16}",
           "ranks": "U{4..40}, sketch width rank + 10", "sampling": "Bernoulli, SR ~ U[0.10, 0.50]",
           "steps": K}
    stream = torch.cuda.Stream()
    res = {}
    for mode in ("sequential", "graph", "graph_autotuned"):
        b = tr.Batch([(p[0], p[1], p[2]) for p in probs], prms,
                     nstreams=1 if mode == "sequential" else 8, stream=stream.cuda_stream)
        if mode == "sequential":
            b.graph_mode(False)
        if not res:
            # turn the generated transform-domain stacks into observed data
            # with each problem's own inverse transform (in place of Xbar)
            for i, p in enumerate(probs):
                h = b.handle(i)
                X = h.transform_inverse(p[0])
                torch.cuda.synchronize()
                p[0].copy_(X * p[1])
                del X
            torch.cuda.synchronize()
        b.step()
        if mode == "graph_autotuned":   # every problem's tube tile and slice split
            t0 = time.perf_counter()
            b.autotune(3)
            tune_s = time.perf_counter() - t0
        b.step()
        torch.cuda.synchronize()
        l0 = b.launches()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(K):
            b.step()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        res[mode] = {"batch_iters_per_s": K / (ms * 1e-3),
                     "problem_iters_per_s": K * len(specs) / (ms * 1e-3),
                     "elements_per_s": K * elems / (ms * 1e-3),
                     "ms_per_batch_iter": ms / K,
                     "kernels_per_batch_iter": (b.launches() - l0) / K,
                     "host_launches_per_batch_iter": 1 if mode != "sequential" else
                     (b.launches() - l0) / K}
        if mode == "graph_autotuned":
            res[mode]["autotune_s"] = tune_s
        b.close()
        torch.cuda.synchronize()
    out.update(res)
    out["graph_vs_sequential"] = res["graph"]["batch_iters_per_s"] / res["sequential"]["batch_iters_per_s"]
    out["autotuned_vs_graph"] = (res["graph_autotuned"]["batch_iters_per_s"]
                                 / res["graph"]["batch_iters_per_s"])
    out["form"] = "%s, 8 streams, one CUDA graph launch per batch iteration" % (
        {0: "fp32 simt", 2: "bf16 tcgen05", 3: "split-bf16 tcgen05"}[prec])
    return out


# ---------------------------------------------------------- reference arm
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2506_09594_gb300 import synth
    w = synth.WORKLOADS[args.workload]
    budget = 150.0
    warm = min(args.warmup, 10)   # oracle iterations take about a second each
    done, el = oracle_steps(args.workload, budget, args.steps, warmup=warm)
    value = done / el
    cores = os.cpu_count() or 1
    sample = ("%d of the %d requested ADMM iterations of %s (numpy float64 oracle, randomized "
              "engine l=%d q=%d), %.1f s" % (done, args.steps, args.workload, w.l, w.q, el))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": done,
        "warmup": warm, "ms_per_step": el / done * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded; tensors shaped like the paper's workloads)",
        "impl": "reference",
        "config": {"workload": args.workload, "dims": list(w.dims), "slices": w.nslices,
                   "rank": w.rank, "sketch_width": w.l, "power_iters": w.q},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def slice_kernels(args):
    """Per-kernel device times of one slice pass of the workload's iterate
    after `warmup` eager steps (few launches, one handle: a case for ncu)."""
    import torch
    from paper_2506_09594_gb300 import synth, tr
    tr.load()
    w = synth.WORKLOADS[args.workload]
    _, M, mask, _ = synth.make_problem(w)
    dt = torch.float64 if w.dtype == "f64" else torch.float32
    Md = torch.from_numpy(M).to("cuda", dt)
    maskd = torch.from_numpy(mask).cuda()
    prec = PREC[args.prec] if w.dtype != "f64" else 0
    stream = torch.cuda.Stream()
    h = make_handle(tr, torch, w, Md, maskd, stream, 0, prec)
    for _ in range(args.warmup):
        h.step()
    s = h.get_state()
    X = (s["L"] + s["Lam"] / s["mu"]).contiguous()
    torch.cuda.synchronize()
    Ab = h.transform_forward(X)
    kern = h.profile_slice_pass(Ab, 1.0 / s["mu"], s["t"], reps=1)
    torch.cuda.synchronize()
    print(json.dumps({"workload": args.workload, "iteration": s["t"], "prec": args.prec,
                      "kernels_us": [[k, ms * 1e3] for k, ms in kern]}))
    h.close()


def main():
    args = parse()
    if args.cpu_child:
        cpu_child(args)
        return
    if args.slice_kernels:
        slice_kernels(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
