#!/usr/bin/env python
"""Benchmark: encrypted KAN inferences/s on GB300.

Workload (one step): the encrypted KAN [4,8,4,1] (grid G=5 on [-1,1], k=3,
SiLU degree 27 on data-fitted ranges) evaluated on a batch of 64 encrypted
inputs (uniform [-1,1]^4) at uneven levels, CKKS N=2^16 with 36 rescaling
levels, one kan_infer call (all 64 inputs in one batched launch sequence).
Inputs stay resident in HBM between steps; one step reads ~2 GB of
ciphertexts plus ~5 GB of switching keys, far above the 129 MB L2.

Reported beside the headline: the per-step p50/p99 latency, HMult/s and
HRot/s at N=2^16 with 37 limbs, the live roofline of the dominant kernel
kind (CUDA events around every launch during the timed region), an
end-to-end figure through the C ABI with pinned host buffers (ciphertexts in,
ciphertexts out, copies inside the timed region), the oracle timed on a
bounded sample on the host cores, and the SM clocks sampled while timing.

Multi-GPU (torchrun): requests shard across ranks (each rank its own batch
and a replica of the keys); no data-path collective, weak scaling.
`--impl reference` times the CPU oracle instead (bounded sample per step).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM bytes (read + write, ncu) over algorithmic bytes of one launch of the
# fused ModUp forward NTT, measured on a 13-limb, batch-8 HMult (the bench's
# launch is too large for a full capture); traffic scales with the units
# processed, so a full launch's traffic is this ratio times its algorithmic
# bytes: 387.7 MB of DRAM traffic (145.5 read, 242.2 written) for 394.3 MB
# algorithmic (13 limbs, 4 digits of 17 rows, batch 8), current kernel build
# (column loads with the source row outermost, grouped epilogue operands).
MODUP_TRAFFIC_RATIO = 387.71 / 394.26

METRIC = "encrypted KAN inferences/s"
UNIT = "inferences/s"
# the configurations: c2 is the headline workload, the others are measured on request
WORKLOADS = {
    "c1": dict(desc="encrypted KAN [2,5,1] G=5 k=3, plain method (one input per launch), CKKS "
                    "N=2^15, q0 + 18 x 40-bit primes, one 60-bit special prime",
               model="kan_2_5_1", inputs="uniform", log_n=15, levels=18, alpha=1, batch=1,
               degree=15, comp=((15,), 0.3), b0="difference", fixed=(-4.0, 4.0), uneven=False),
    "c2": dict(desc="encrypted KAN [4,8,4,1] G=5 k=3, CKKS N=2^16, 36 levels, batch 64 "
                    "(input levels over the chain's spare levels: none at this accuracy)",
               model="kan_4_8_4_1", inputs="uniform", log_n=16, levels=36, alpha=0, batch=64,
               degree=27, comp=((7, 15), 0.12), b0="difference", fixed=None, uneven=True),
    "c3": dict(desc="encrypted KAN [784,64,10] G=5 k=3 on synthetic 28x28 blob images, CKKS "
                    "N=2^16, 36 levels, batch 32",
               model="kan_784_64_10", inputs="blob", log_n=16, levels=36, alpha=0, batch=32,
               degree=15, comp=((7, 7, 7), 0.05), b0="product", fixed=None, uneven=False),
    "c4": dict(desc="encrypted KAN [3072,64,10] G=10 k=3 on synthetic 3x32x32 images (two "
                    "ciphertexts per image), CKKS N=2^16, 36 levels, batch 16",
               model="kan_3072_64_10", inputs="cifar", log_n=16, levels=36, alpha=0, batch=16,
               degree=15, comp=((7, 7, 15), 0.03), b0="product", fixed=None, uneven=False),
}
WORKLOAD = WORKLOADS["c2"]["desc"]


def args_():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--batch", type=int, default=64)
    p.add_argument("--log-n", type=int, default=16)
    p.add_argument("--levels", type=int, default=36)
    p.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-micro", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the other configurations (C1, C3, C4, C5 serving, Table 3 shapes) "
                        "that the default run measures after the headline")
    p.add_argument("--kernel", default=None, choices=["ntt", "intt", "hmult"],
                   help="time one kernel kind alone (NTT limbs/s) instead of the network")
    p.add_argument("--rows", type=int, default=592, help="limbs per launch for --kernel")
    p.add_argument("--serve", action="store_true",
                   help="Poisson serving mix through the continuous-batching server")
    p.add_argument("--graphs", action="store_true",
                   help="time CUDA-graph replays of the layer schedules instead of eager launches")
    p.add_argument("--alpha", type=int, default=0,
                   help="key-switching digit size (special primes); 0 = autotune within --max-qp-bits")
    p.add_argument("--p-bits", type=int, default=60,
                   help="special prime size when --alpha is given (alpha 5 needs 48 within the "
                        "1740-bit bound)")
    p.add_argument("--max-qp-bits", type=int, default=1740,
                   help="bound on log2(QP) for the digit-layout autotuner (128-bit budget)")
    p.add_argument("--workload", default="c2", choices=sorted(WORKLOADS),
                   help="configuration to time (c2, the default, is the headline workload; "
                        "sets log-n, levels, batch and alpha)")
    p.add_argument("--table3", action="store_true",
                   help="one KAN layer per (n_i, g, k) shape: lazy combination vs the naive method")
    p.add_argument("--oracle-micro", action="store_true",
                   help="with --impl reference: also time the oracle's NTT per limb, HMult and "
                        "HRot at the top level (single thread; about a minute)")
    p.add_argument("--bsgs", default="single", choices=["single", "double"],
                   help="BSGS form of the KAN layers' matvecs (hoisted or double-hoisted)")
    p.add_argument("--boot", action="store_true", help="time CKKS bootstrapping at N=2^16")
    p.add_argument("--deep", action="store_true",
                   help="time a five-layer KAN refreshed by bootstrapping between layers")
    p.add_argument("--boot-batch", type=int, default=8)
    p.add_argument("--boot-form", default="double", choices=["single", "double"])
    p.add_argument("--rate", type=float, default=20.0, help="requests/s for --serve")
    p.add_argument("--duration", type=float, default=10.0, help="seconds of arrivals for --serve")
    return p.parse_args()


TABLE3_SHAPES = [(64, 3, 2), (128, 5, 3), (256, 5, 3), (256, 10, 3), (256, 10, 5)]


def table3_arm(a):
    """--table3: the B-spline layer shapes (n_i, g, k) of the paper's Table 3,
    each as one KAN layer [n_i, 64] (SiLU degree 15, comparison f_3) on one
    encrypted input at N=2^16 with 14 levels: kan_layer_eval with lazy
    combination (W_f = W'P, Eq. 13) against the naive method (HE permutation
    by P, then W'). Reports GPU ms per layer and the plaintext-multiply and
    rotation launches of each schedule."""
    import numpy as np
    import torch
    from paper_2409_07751_gb300 import build
    build.build()
    from paper_2409_07751_gb300 import ckks as G
    from paper_2409_07751_gb300 import workloads as W
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = G.Context(a.log_n, 14, 4)
    ctx.set_stream(stream.cuda_stream)
    rows = []
    for n_i, g, k in TABLE3_SHAPES:
        model = W.make_model("t", widths=[n_i, 64], G=g, k=k)
        X = W.uniform_inputs(65, n_i)
        m = G.calibrate(model, X[1:], 15, [3])
        row = {"n_i": n_i, "g": g, "k": k, "n_out": 64}
        for naive in (False, True):
            gm = G.Model(ctx, [dict(L, naive=naive) for L in m])
            keys = G.Keys(ctx, W.SEED_KEYS, gm.rotations())
            x = G.encrypt(ctx, keys, X[:1], 14, W.SEED_ENC, 0)
            G.kan_layer_eval(ctx, keys, gm, 0, x).close()  # plaintext cache
            torch.cuda.synchronize()
            before = ctx.launch_counts()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 3
            e0.record(stream)
            for _ in range(reps):
                G.kan_layer_eval(ctx, keys, gm, 0, x).close()
            e1.record(stream)
            torch.cuda.synchronize()
            after = ctx.launch_counts()
            tag = "naive" if naive else "lazy"
            row[tag + "_ms"] = e0.elapsed_time(e1) / reps
            row[tag + "_mul_plain"] = (after["mul_plain"] - before["mul_plain"]) // reps
            row[tag + "_rotations"] = (after["rotate_finish"] - before["rotate_finish"]) // reps
            row[tag + "_depth"] = gm.layer_depth(0)
            x.close()
            keys.close()
            gm.close()
        row["speedup"] = row["naive_ms"] / row["lazy_ms"]
        rows.append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps({"metric": "KAN layer latency, lazy combination vs naive (Table 3 shapes)",
                      "unit": "ms", "n_poly": 1 << a.log_n, "levels": 14, "batch": 1,
                      "rows": rows}), flush=True)


def serve_arm(a):
    """--serve: Poisson arrivals (rate/s for `duration` s) of a mix of 50 %
    [2,5,1], 30 % [784,64,10] and 20 % [3072,64,10] requests, one key set per
    model (a simulated client each), all at N=2^16 / 36 levels; requests are
    encrypted on arrival and submitted to the native server, which steps
    continuously. Latency = arrival to finished ciphertext."""
    import numpy as np
    import torch
    from paper_2409_07751_gb300 import build
    build.build()
    from paper_2409_07751_gb300 import ckks as G
    from paper_2409_07751_gb300 import workloads as W
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    alpha, p_bits = a.alpha, 60
    if alpha == 0:
        alpha, p_bits, _ = G.autotune_keyswitch(a.log_n, a.levels, a.max_qp_bits, batch=8)
    ctx = G.Context(a.log_n, a.levels, alpha, p_bits=p_bits)
    ctx.set_stream(stream.cuda_stream)
    # every model at the chain's 36 levels with two layers: the four-stage
    # degree-7 minimax comparison (eps 0.02) in Algorithm 2's product form
    stages = G.comp_minimax(0.02, (7, 7, 7, 7))[0]
    specs = [("kan_2_5_1", lambda n, s: W.uniform_inputs(n, 2, seed=s), 15, stages, (-4.0, 4.0), 0.5),
             ("kan_784_64_10", lambda n, s: W.blob_images(n, seed=s), 15, stages, None, 0.3),
             ("kan_3072_64_10", lambda n, s: W.cifar_like_images(n, seed=s), 15, stages, None,
              0.2)]
    srv = G.Server(ctx, int(200e9))
    models = []
    for i, (name, gen, deg, comp, fr, share) in enumerate(specs):
        m = G.calibrate(W.make_model(name), gen(64, W.SEED_INPUTS + 1000), deg, comp, fixed_range=fr)
        gm = G.Model(ctx, m)
        keys = G.Keys(ctx, W.SEED_KEYS + i, gm.rotations())
        models.append((srv.add_model(gm, keys), gm, keys, gen, share))
    arrivals = W.poisson_arrivals(a.rate, a.duration)
    pick = np.random.default_rng(W.SEED_ARRIVALS + 1).choice(
        len(models), size=len(arrivals), p=[mm[4] for mm in models])

    def request(i):
        mid, gm, keys, gen, _ = models[pick[i]]
        x = gm.pack_input(gen(1, W.SEED_INPUTS + 10000 + i)[0])
        return mid, G.encrypt(ctx, keys, x, a.levels, W.SEED_ENC, 64 * i)

    # warm-up: one request of each model end to end (plaintext caches, code paths)
    for j in range(len(models)):
        mid, ct = request(int(np.nonzero(pick == j)[0][0]))
        rid = srv.submit(mid, ct)
        while srv.take(rid) is None:
            srv.step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pending, lat, nxt = {}, [], 0
    while nxt < len(arrivals) or pending:
        now = time.perf_counter() - t0
        while nxt < len(arrivals) and arrivals[nxt] <= now:
            mid, ct = request(nxt)
            pending[srv.submit(mid, ct)] = (arrivals[nxt], int(pick[nxt]))
            nxt += 1
        if not pending:
            time.sleep(max(0.0, min(0.01, arrivals[nxt] - now)))
            continue
        srv.step()
        torch.cuda.synchronize()
        done = time.perf_counter() - t0
        for rid in list(pending):
            out = srv.take(rid)
            if out is not None:
                t_arr, which = pending.pop(rid)
                lat.append((t_arr, done - t_arr, which))
                out.close()
    wall = time.perf_counter() - t0
    st = srv.status()
    warm = 5.0 if a.duration > 10.0 else 0.0  # arrivals in the first 5 s are warm-up
    kept = [l for t, l, _ in lat if t >= warm]
    names = [sp[0] for sp in specs]
    per_model = {}
    for j, name in enumerate(names):
        lj = [l for t, l, w in lat if w == j and t >= warm]
        per_model[name] = {"requests": len([1 for _, _, w in lat if w == j]),
                           "p50_ms": 1000 * float(np.percentile(lj, 50)) if lj else None}

    # the plain form on the same request mix: one request at a time through
    # kan_infer, no batching across requests
    n_plain = min(40, len(arrivals))
    torch.cuda.synchronize()
    tp = time.perf_counter()
    for i in range(n_plain):
        mid, ct = request(i)
        _, gm_i, keys_i, _, _ = models[pick[i]]
        G.kan_infer(ctx, keys_i, gm_i, [ct]).close()
        torch.cuda.synchronize()
    plain_rate = n_plain / (time.perf_counter() - tp)
    print(json.dumps({
        "metric": "encrypted KAN inferences/s (serving mix)", "value": len(lat) / wall,
        "unit": UNIT, "higher_is_better": True, "n_gpus": 1, "dtype": "u64", "data": "synthetic",
        "latency_ms": {"p50": 1000 * float(np.percentile(kept, 50)),
                       "p99": 1000 * float(np.percentile(kept, 99)),
                       "excluded_warmup_s": warm, "requests_counted": len(kept)},
        "requests": len(lat), "wall_s": wall, "hbm_peak_bytes": st["hbm_measured_peak"],
        "hbm_peak_admitted_bytes": st["hbm_peak"], "hbm_budget_bytes": int(200e9),
        "admission": {"footprint_bytes_per_request": {sp[0]: srv.footprint(mm[0])
                                                      for sp, mm in zip(specs, models)},
                      "how": "measured per model at kan_server_add_model (device pool "
                             "watermark over one network run at the top level); hbm_peak_bytes "
                             "is the largest rise of the pool's used bytes over one step"},
        "per_model": per_model,
        "plain_form": {"value": plain_rate, "unit": UNIT, "requests": n_plain,
                       "how": "one request at a time through kan_infer, same mix"},
        "config": {"workload": "Poisson serving mix", "rate_per_s": a.rate, "duration_s": a.duration,
                   "mix": {"kan_2_5_1": 0.5, "kan_784_64_10": 0.3, "kan_3072_64_10": 0.2},
                   "n_poly": 1 << a.log_n, "levels": a.levels, "alpha": alpha,
                   "p_bits": p_bits}}), flush=True)


def kernel_arm(a):
    """--kernel ntt|intt: forward or inverse NTT of `rows` random limbs of
    N = 2^log_n (moduli cycling through the Q primes) per launch;
    --kernel hmult: HMult with relinearisation and rescale of `batch`
    ciphertexts at the top level."""
    import numpy as np
    import torch
    from paper_2409_07751_gb300 import build
    build.build()
    from paper_2409_07751_gb300 import ckks as G
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = G.Context(a.log_n, a.levels, 4)
    ctx.set_stream(stream.cuda_stream)
    limbs = a.levels + 1
    N = 1 << a.log_n
    if a.kernel == "hmult":
        # HMult (tensor, ModUp, key inner product, ModDown, rescale) on a
        # batch of `batch` ciphertexts at the top level
        keys = G.Keys(ctx, 1, [])
        x = G.encrypt(ctx, keys, np.random.default_rng(0).uniform(-1, 1, (a.batch, ctx.slots)),
                      a.levels, 2, 0)
        for _ in range(a.warmup):
            G.mul(ctx, keys, x, x).close()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            G.mul(ctx, keys, x, x).close()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.steps
        print(json.dumps({"kernel": "hmult", "batch": a.batch, "limbs": limbs, "n_poly": N,
                          "ms_per_call": ms, "hmult_per_s": a.batch / (ms / 1000.0)}), flush=True)
        return
    rng = np.random.default_rng(0)
    h = np.stack([rng.integers(0, int(ctx.moduli[r % limbs]), N, dtype=np.uint64) for r in range(a.rows)])
    d = torch.from_numpy(h.view(np.int64)).cuda()
    inv = a.kernel == "intt"
    for _ in range(a.warmup):
        ctx.ntt(d.data_ptr(), a.rows, limbs, inv)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        ctx.ntt(d.data_ptr(), a.rows, limbs, inv)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    by = 2.0 * a.rows * N * 8
    print(json.dumps({"kernel": a.kernel, "rows": a.rows, "n_poly": N, "ms_per_launch": ms,
                      "limbs_per_s": a.rows / (ms / 1000.0), "algorithmic_GBps": by / (ms / 1000.0) / 1e9}),
          flush=True)


BOOT_DESC = ("CKKS bootstrapping (ModRaise, CoeffToSlot, EvalMod, SlotToCoeff) of full-slot "
             "ciphertexts, N=2^16, 60-bit q0 + 28 x 50-bit primes, 5 x 60-bit special primes "
             "(log QP 1760), sparse secret h=192, |I| <= 30, EvalMod degree 255, 3 + 3 merged "
             "transform levels, double-hoisted transforms")


def boot_arm(a):
    """--boot: bootstraps/s of a batch of `boot_batch` level-0 ciphertexts
    refreshed in one call (inputs resident), the batch-1 latency, the
    refreshed slots' error, and the live roofline of the dominant kernel kind
    (per-launch CUDA events over a profiled repeat)."""
    import numpy as np
    import torch
    from paper_2409_07751_gb300 import build
    build.build()
    from paper_2409_07751_gb300 import ckks as G
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = G.Context(16, 28, 5, q0_bits=60, scale_bits=50)
    ctx.set_stream(stream.cuda_stream)
    t0 = time.perf_counter()
    plan = G.BootPlan(ctx, 30, 255, 3, 3, form=a.boot_form)
    keys = G.Keys(ctx, 7, plan.rotations(), hamming_weight=192, conjugation=True)
    ctx.synchronize()
    setup_s = time.perf_counter() - t0
    B = a.boot_batch
    z = np.random.default_rng(6).uniform(-1, 1, (B, ctx.slots))
    ct = G.encrypt(ctx, keys, z, 0, 9, 0)
    out = plan.bootstrap(keys, ct)
    err = float(np.abs(G.decrypt(ctx, keys, out, ctx.slots) - z).max())
    level = out.level
    out.close()
    for _ in range(a.warmup):
        plan.bootstrap(keys, ct).close()
    torch.cuda.synchronize()
    before = ctx.launch_counts()
    clk = Clocks(torch.cuda.current_device())
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    ev[0].record(stream)
    for i in range(a.steps):
        plan.bootstrap(keys, ct).close()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    after = ctx.launch_counts()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(a.steps)]
    ms = ev[0].elapsed_time(ev[-1]) / a.steps
    launches = sum(after[k] - before[k] for k in after if k != "copy") // a.steps
    ctx.profile(True)
    plan.bootstrap(keys, ct).close()
    torch.cuda.synchronize()
    prof = ctx.profile_collect()
    ctx.profile(False)
    kinds = {k: v for k, v in prof.items() if k != "copy"}
    total = sum(v[0] for v in kinds.values())
    dom = max(kinds, key=lambda k: kinds[k][0])
    kms, kby, kn, kmm = kinds[dom]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = kby / (kms / 1000.0) / 1e9
    bpk = ctx.int_peak(1) / 1e9
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "algorithmic_bytes_per_launch": kby / kn, "avg_launch_ms": kms / kn,
                "share_of_kernel_time": kms / total}
    if kmm > 0:
        alu = kmm / (kms / 1000.0) / 1e9
        roofline["alu"] = {"achieved": alu, "unit": "G modmul/s", "peak": bpk, "frac": alu / bpk,
                           "peak_source": "measured: register-only lazy forward butterflies"}
    lat = []
    one = G.encrypt(ctx, keys, z[:1], 0, 9, 0)
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.bootstrap(keys, one).close()
        e1.record(stream)
        torch.cuda.synchronize()
        lat.append(e0.elapsed_time(e1))
    print(json.dumps({
        "metric": "CKKS bootstraps/s", "value": B / (ms / 1000.0), "unit": "bootstraps/s",
        "ms_per_step": ms, "steps": a.steps, "warmup": a.warmup, "batch": B,
        "latency_ms_batch1": min(lat), "max_abs_error": err, "output_level": level,
        "gpu_launches_per_step": launches, "setup_s": round(setup_s, 2),
        "step_ms": [round(x, 2) for x in step_ms], "roofline": roofline,
        "kernel_time_shares": {k: round(v[0] / total, 4)
                               for k, v in sorted(kinds.items(), key=lambda kv: -kv[1][0])[:8]},
        "clocks": clocks, "dtype": "u64", "data": "synthetic",
        "config": {"workload": BOOT_DESC, "form": a.boot_form, "rotation_keys": len(plan.rotations()),
                   "l2": "inputs and keys (several GB) far above L2"}}), flush=True)


DEEP_DESC = ("encrypted KAN [4,8,8,8,4,1] G=5 k=3 (SiLU degree 27, minimax comparison degrees 7 "
             "and 15, eps 0.12, difference form: 12 levels per layer, 60 in all), CKKS N=2^16, "
             "60-bit q0 + 29 x 50-bit primes, 4 x 60-bit special primes (log QP 1750), the batch "
             "refreshed before layers 3, 4 and 5 (masked, packed into one ciphertext, one "
             "bootstrap with 2 + 3 merged transform levels, unpacked)")


def deep_arm(a):
    """--deep: a KAN deeper than any leveled chain inside the security budget,
    run by kan_infer with a bootstrapping plan set (the batch refreshed
    packed when the next layer needs more levels than are left); inferences/s
    of a batch, and beside it the time bootstrapping the batch ciphertext by
    ciphertext takes (the unpacked refresh)."""
    import numpy as np
    import torch
    from paper_2409_07751_gb300 import build
    build.build()
    from paper_2409_07751_gb300 import ckks as G, workloads as W
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = G.Context(16, 29, 4, q0_bits=60, scale_bits=50)
    ctx.set_stream(stream.cuda_stream)
    t0 = time.perf_counter()
    model = [dict(L, b0="difference") for L in W.make_model("t", widths=[4, 8, 8, 8, 4, 1], G=5, k=3)]
    Xcal = W.uniform_inputs(256, 4, seed=W.SEED_INPUTS + 1000)
    m = G.calibrate(model, Xcal, 27, G.comp_minimax(0.12, (7, 15))[0])
    gm = G.Model(ctx, m)
    depths = [gm.layer_depth(i) for i in range(len(m))]
    plan = G.BootPlan(ctx, 30, 255, 2, 3)
    keys = G.Keys(ctx, 7, sorted(set(gm.rotations()) | set(plan.rotations())
                                 | set(gm.refresh_rotations(a.batch))),
                  hamming_weight=192, conjugation=True)
    gm.set_bootstrap(plan)
    x = W.uniform_inputs(a.batch, 4)
    ct = G.encrypt(ctx, keys, x, ctx.L, W.SEED_ENC, 0)
    ctx.synchronize()
    setup_s = time.perf_counter() - t0
    out = G.kan_infer(ctx, keys, gm, [ct])
    level = out.level
    out.close()
    for _ in range(a.warmup):
        G.kan_infer(ctx, keys, gm, [ct]).close()
    torch.cuda.synchronize()
    clk = Clocks(torch.cuda.current_device())
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    ev[0].record(stream)
    for i in range(a.steps):
        G.kan_infer(ctx, keys, gm, [ct]).close()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = ev[0].elapsed_time(ev[-1]) / a.steps
    # bootstrapping every ciphertext of the batch (the unpacked refresh)
    low = G.level_down(ctx, ct, 0)
    plan.bootstrap(keys, low).close()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.bootstrap(keys, low).close()
    e1.record(stream)
    torch.cuda.synchronize()
    refresh_ms = e0.elapsed_time(e1)
    lv, refreshes = ctx.L, 0
    for i, d in enumerate(depths):
        if i > 0 and lv < d:
            lv, refreshes = plan.stc_level - 3, refreshes + 1
        lv -= d
    # packed refreshes: one bootstrap per N/2 / 8 ciphertexts (the 8-slot block)
    boots_per_refresh = -(-a.batch // (ctx.slots // 8))
    print(json.dumps({
        "metric": "encrypted KAN inferences/s (bootstrapped)", "value": a.batch / (ms / 1000.0),
        "unit": "inferences/s", "ms_per_step": ms, "steps": a.steps, "warmup": a.warmup,
        "batch": a.batch, "layer_depths": depths, "refreshes_per_batch": refreshes,
        "bootstraps_per_refresh": boots_per_refresh,
        "bootstrap_ms_per_ciphertext_batch": refresh_ms, "output_level": level,
        "setup_s": round(setup_s, 1), "clocks": clocks, "dtype": "u64", "data": "synthetic",
        "config": {"workload": DEEP_DESC, "batch_per_gpu": a.batch,
                   "l2": "inputs and keys (tens of GB) far above L2"}}), flush=True)


def config(a):
    wl = workload(a)
    return {"workload": wl["desc"], "model": wl["model"], "n_poly": 1 << a.log_n,
            "levels": a.levels, "batch_per_gpu": a.batch, "silu_degree": wl["degree"],
            "comparison": "minimax composite, stage degrees %s, eps %g, B_{m,0} %s form"
                          % ("-".join(str(d) for d in wl["comp"][0]), wl["comp"][1], wl["b0"]),
            "input_levels": "uniform over [L - slack, L]" if wl["uneven"]
                            else "all at the network's depth (<= L)",
            "parallelism": "replicas (request sharding)",
            "l2": "inputs larger than L2 (ciphertexts + keys per step >> 129 MB)",
            "schedule": "CUDA graph per layer" if getattr(a, "graphs", False) else "eager",
            "bsgs": getattr(a, "bsgs", "single"),
            "alpha": getattr(a, "alpha", 4), "p_bits": getattr(a, "p_bits", 60),
            "log_qp": 60 + 40 * a.levels + getattr(a, "alpha", 4) * getattr(a, "p_bits", 60)}


def shard_plan(rank, batch):
    """Request sharding across ranks: rank r serves its own batch (its own
    input and level seeds, object ids r*batch ..), with no exchange."""
    from paper_2409_07751_gb300 import workloads as W
    return {"input_seed": W.SEED_INPUTS + rank, "level_seed": W.SEED_INPUTS + 1 + rank,
            "first_index": rank * batch}


def reduce_max(value, dist, device):
    """Max of a per-rank scalar over all ranks (the slowest rank sets the time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(a):
    return WORKLOADS[getattr(a, "workload", "c2")]


def model_and_inputs(a, rank):
    from paper_2409_07751_gb300 import workloads as W
    wl = workload(a)
    model = [dict(L, b0=wl["b0"], bsgs=a.bsgs) for L in W.make_model(wl["model"])]
    n_in = model[0]["n_in"]
    gen = {"uniform": lambda n, s: W.uniform_inputs(n, n_in, seed=s),
           "blob": lambda n, s: W.blob_images(n, seed=s),
           "cifar": lambda n, s: W.cifar_like_images(n, seed=s)}[wl["inputs"]]
    Xcal = gen(256 if wl["inputs"] == "uniform" else 64, W.SEED_INPUTS + 1000)
    X = gen(a.batch, shard_plan(rank, a.batch)["input_seed"])
    return model, Xcal, X


def calibrate_for(a, calibrate, model, Xcal, design):
    """The model's HE parameters: the comparison composite from `design`
    (eps, degrees) -> stages, then calibrate(...)."""
    wl = workload(a)
    degs, eps = wl["comp"]
    stages = design(eps, degs)
    return calibrate(model, Xcal, wl["degree"], stages, fixed_range=wl["fixed"])


def gpu_design(G):
    return lambda eps, degs: G.comp_minimax(eps, degs)[0]


def oracle_design(eps, degs):
    from oracle import polycomp
    return polycomp.composite(eps, degs)[0]


# ------------------------------------------------------------------ clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(device)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle sample
def oracle_sample(model_he, a, budget_s, steps=1, warmup=0):
    """Time the oracle (plain single-threaded CPU code) on the same workload.

    The oracle needs minutes to hours per inference at N=2^16, so each sample
    runs one inference from the start and stops after `budget_s` seconds at a
    key-switch boundary; the fraction done is the number of key switches
    completed over the inference's total (counted on the same schedule at
    N=2^11, where the rotation plans are identical). Keys and the input are
    random residues of the right shapes (timing does not depend on them).
    """
    import numpy as np
    from oracle import ckks as O, kan_he

    class _Stop(Exception):
        pass

    real_ks, real_ksr, real_modup = O._ks, O._ks_rescale, O._modup

    # the key switches of one inference and their levels (same schedule,
    # small ring, no arithmetic)
    counter = {"levels": []}

    def count_ks(ctx, ext, level, key, g):
        counter["levels"].append(level)
        return np.zeros((2, level + 1, ctx.N), np.uint64)

    def count_ksr(ctx, d, ext, level, key):
        counter["levels"].append(level)
        return np.zeros((2, level, ctx.N), np.uint64)

    def skip_modup(ctx, poly, level):
        return None

    # the [2,5,1] and [4,8,4,1] schedules are the same at N = 2^11; the image
    # models' packing and chunking depend on the ring, so they count on theirs
    small = O.Ctx(O.Params(11 if workload(a)["model"] in ("kan_2_5_1", "kan_4_8_4_1") else a.log_n,
                           a.levels, 4))

    class Fake:
        pass

    fk = Fake()
    fk.relin = None
    fk.galois = {small.galois(t): None for t in kan_he.model_rotations(model_he, small.slots)}
    x = O.Ct(np.zeros((2, a.levels + 1, small.N), np.uint64), a.levels, small.delta[a.levels])
    K = kan_he.chunking(model_he[0], small.slots)[0]
    if K > 1:
        x = [x] * K
    O._ks, O._ks_rescale, O._modup = count_ks, count_ksr, skip_modup
    try:
        kan_he.infer(small, fk, x, model_he)
    finally:
        O._ks, O._ks_rescale, O._modup = real_ks, real_ksr, real_modup
    total = len(counter["levels"])
    ctx = O.Ctx(O.Params(a.log_n, a.levels, getattr(a, "alpha", 0) or 4, p_bits=getattr(a, "p_bits", 60)))

    def weight(level):
        # transforms of one key switch at `level` (l limbs, beta digits):
        # ModUp's l inverse and beta (l + alpha) - l forward, ModDown's
        # 2 alpha inverse and 2 l forward; the schedule's other work (rescales,
        # plaintext products) also grows with l and is timed inside the sample
        l, A = level + 1, ctx.alpha
        beta = -(-l // A)
        return l + beta * (l + A) - l + 2 * A + 2 * l

    total_w = sum(weight(lv) for lv in counter["levels"])

    Z = np.zeros((ctx.beta_max, 2, ctx.n_qp, ctx.N), np.uint64)
    keys = Fake()
    keys.relin = Z
    keys.galois = {ctx.galois(t): Z for t in kan_he.model_rotations(model_he, ctx.slots)}
    rng = np.random.default_rng(0)
    data = np.stack([np.stack([rng.integers(0, ctx.q[t], ctx.N, dtype=np.uint64)
                               for t in range(a.levels + 1)]) for _ in range(2)])
    ct = O.Ct(data, a.levels, ctx.delta[a.levels])
    K = kan_he.chunking(model_he[0], ctx.slots)[0]
    if K > 1:
        ct = [ct] * K
    rates = []
    for it in range(warmup + steps):
        done = {"n": 0, "w": 0.0}
        t0 = time.perf_counter()

        def tick(level):
            done["n"] += 1
            done["w"] += weight(level)
            if time.perf_counter() - t0 > budget_s:
                raise _Stop()

        def timed_ks(ctx_, ext, level, key, g):
            r = real_ks(ctx_, ext, level, key, g)
            tick(level)
            return r

        def timed_ksr(ctx_, d, ext, level, key):
            r = real_ksr(ctx_, d, ext, level, key)
            tick(level)
            return r

        O._ks, O._ks_rescale = timed_ks, timed_ksr
        try:
            kan_he.infer(ctx, keys, ct, model_he)
        except _Stop:
            pass
        finally:
            O._ks, O._ks_rescale = real_ks, real_ksr
        el = time.perf_counter() - t0
        if it >= warmup:
            rates.append((done["w"] / total_w) / el)
    sample = ("first %d of %d key switches of one inference (N=2^%d, %d levels), single thread, "
              "random keys and input, %.0f s budget per sample; fraction done = their share of the "
              "schedule's key-switch transforms weighted by level (%.4f)"
              % (done["n"], total, a.log_n, a.levels, budget_s, done["w"] / total_w))
    return statistics.mean(rates), sample, total


def c1_oracle_full():
    """One whole encrypted [2,5,1] inference by the oracle, single thread, at
    its full size (N=2^15, q0 + 18 x 40-bit primes, one special prime):
    seconds for kan_he.infer alone (keys and the encryption made first)."""
    from oracle import calibrate as OC, ckks as O, kan_he
    from paper_2409_07751_gb300 import workloads as W
    wl = WORKLOADS["c1"]
    model = W.make_model(wl["model"])
    Xcal = W.uniform_inputs(256, 2, seed=W.SEED_INPUTS + 1000)
    model = [dict(L, b0=wl["b0"]) for L in model]
    m = OC.calibrate(model, Xcal, wl["degree"], oracle_design(wl["comp"][1], wl["comp"][0]),
                     fixed_range=wl["fixed"])
    ctx = O.Ctx(O.Params(wl["log_n"], wl["levels"], wl["alpha"]))
    keys = O.Keys(ctx, W.SEED_KEYS, kan_he.model_rotations(m, ctx.slots))
    x = O.encrypt(ctx, keys, W.uniform_inputs(1, 2)[0], wl["levels"], W.SEED_ENC, 0)
    t0 = time.perf_counter()
    kan_he.infer(ctx, keys, x, m)
    return time.perf_counter() - t0


def _oracle_worker(job):
    m, a, budget, steps, warmup = job
    return oracle_sample(m, a, budget, steps=steps, warmup=warmup)[:2]


def oracle_all_cores(m, a, budget, steps=1, warmup=0, procs=None):
    """The oracle on every host core: independent inferences in `procs`
    spawned processes (the oracle is single-threaded), each a bounded
    sample; the rate is the sum over processes."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(m, a, budget, steps, warmup)] * procs)
    return sum(r for r, _ in res), res[0][1], procs


def reference_arm(a):
    """--impl reference: the CPU oracle as it stands, bounded samples."""
    from paper_2409_07751_gb300 import workloads as W
    from oracle import calibrate as OC
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # the digit layout the GPU arm's autotuner selects on GB300 (alpha = 5,
    # 48-bit special primes); the oracle cannot run the timing itself
    if not a.alpha:
        a.alpha, a.p_bits = 5, 48
    model, Xcal, _ = model_and_inputs(a, 0)
    m = calibrate_for(a, OC.calibrate, model, Xcal, oracle_design)
    per_step = max(5.0, min(a.cpu_budget, 150.0 / max(1, a.steps + a.warmup)))
    t0 = time.perf_counter()
    v, sample, procs = oracle_all_cores(m, a, per_step, steps=a.steps, warmup=a.warmup)
    sample = "%d processes, each: %s" % (procs, sample)
    el = time.perf_counter() - t0
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000.0 * el / (a.steps + a.warmup),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": config(a),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if a.oracle_micro:
        line["oracle_micro"] = oracle_micro(a)
    print(json.dumps(line), flush=True)


def oracle_micro(a):
    """Single-threaded oracle op times at the workload's ring and top level,
    in the digit layout of the reference arm: forward and inverse NTT per
    limb, HMult (tensor, merged relinearise-rescale) and HRot of one
    ciphertext. Keys and inputs are seeded; one run of each op."""
    import numpy as np
    from oracle import ckks as O
    ctx = O.Ctx(O.Params(a.log_n, a.levels, a.alpha, p_bits=a.p_bits))
    keys = O.Keys(ctx, 7, [1])
    v = np.random.default_rng(5).uniform(-1, 1, ctx.slots)
    x = O.encrypt(ctx, keys, v, a.levels, 9, 0)
    limbs = a.levels + 1
    rows = np.random.default_rng(6).integers(0, 2**39, (limbs, 1 << a.log_n), dtype=np.uint64)
    out = {"n_poly": 1 << a.log_n, "limbs": limbs, "alpha": a.alpha, "p_bits": a.p_bits,
           "threads": 1}
    for name, inv in (("ntt_ms_per_limb", 0), ("intt_ms_per_limb", 1)):
        t0 = time.perf_counter()
        for t in range(limbs):
            ctx.L_.or_ntt_limb(ctx.h, rows[t].ctypes.data, t, inv)
        out[name] = 1000.0 * (time.perf_counter() - t0) / limbs
    t0 = time.perf_counter()
    O.mul(ctx, keys, x, x)
    out["hmult_ms"] = 1000.0 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    O.rotate(ctx, keys, x, 1)
    out["hrot_ms"] = 1000.0 * (time.perf_counter() - t0)
    return out


# ------------------------------------------------------------------ other configurations
EXTRA_RUNS = [
    ("c1", ["--workload", "c1", "--steps", "20", "--warmup", "3", "--graphs"], 300),
    ("c3", ["--workload", "c3", "--steps", "3", "--warmup", "3"], 600),
    ("c4", ["--workload", "c4", "--steps", "3", "--warmup", "3"], 600),
    ("c5_serve", ["--serve", "--rate", "20", "--duration", "30"], 900),
    ("c5_serve_10", ["--serve", "--rate", "10", "--duration", "30"], 900),
    ("table3", ["--table3"], 600),
    ("boot", ["--boot", "--steps", "3", "--warmup", "2"], 600),
    ("deep_kan", ["--deep", "--batch", "32", "--steps", "2", "--warmup", "1"], 900),
]


def _summary(name, line):
    if "error" in line:
        return line
    if name in ("c1", "c3", "c4"):
        return {k: line.get(k) for k in ("value", "unit", "ms_per_step", "steps", "warmup",
                                           "latency_ms", "depth", "clocks")} | {
            "batch": line["config"]["batch_per_gpu"], "workload": line["config"]["workload"],
            "alpha": line["config"]["alpha"], "p_bits": line["config"]["p_bits"],
            "dominant_kernel": {k: line["roofline"].get(k) for k in ("kernel", "frac", "unit")}}
    if name == "deep_kan":
        return {k: line.get(k) for k in ("value", "unit", "ms_per_step", "batch", "layer_depths",
                                           "refreshes_per_batch", "bootstraps_per_refresh",
                                           "bootstrap_ms_per_ciphertext_batch", "clocks",
                                           "config")}
    if name == "boot":
        return {k: line.get(k) for k in ("value", "unit", "ms_per_step", "batch", "latency_ms_batch1",
                                           "max_abs_error", "output_level", "gpu_launches_per_step",
                                           "kernel_time_shares", "clocks", "config")} | {
            "dominant_kernel": {k: line["roofline"].get(k) for k in ("kernel", "frac", "unit")}}
    if name in ("c5_serve", "c5_serve_10"):
        return {k: line.get(k) for k in ("value", "unit", "latency_ms", "requests", "wall_s",
                                           "hbm_peak_bytes", "hbm_budget_bytes", "admission",
                                           "plain_form", "per_model", "config")}
    return {"rows": [{k: r[k] for k in ("n_i", "g", "k", "lazy_ms", "naive_ms", "speedup")}
                     for r in line.get("rows", [])], "unit": "ms per layer",
            "levels": line.get("levels"), "n_poly": line.get("n_poly")}


def extras(device):
    """The other configurations, each a short child run of this script on
    the same GPU (its own context, keys and models), summarised; the SM clocks
    are sampled over the whole phase."""
    out = {}
    clk = Clocks(device)
    t0 = time.perf_counter()
    for name, args, limit in EXTRA_RUNS:
        cmd = [sys.executable, os.path.join(ROOT, "bench.py")] + args
        if name in ("c1", "c3", "c4"):
            cmd += ["--no-micro", "--no-e2e", "--no-cpu-baseline", "--no-extras"]
        t = time.perf_counter()
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=limit)
            lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
            if r.returncode == 0 and lines:
                line = json.loads(lines[-1])
            else:
                line = {"error": "rc %d: %s" % (r.returncode, r.stderr[-400:])}
        except subprocess.TimeoutExpired:
            line = {"error": "did not finish within %d s" % limit}
        out[name] = _summary(name, line)
        out[name]["wall_s"] = round(time.perf_counter() - t, 1)
    out["clocks"] = clk.stop()
    out["wall_s"] = round(time.perf_counter() - t0, 1)
    out["how"] = " ; ".join("%s: bench.py %s" % (n, " ".join(a)) for n, a, _ in EXTRA_RUNS)
    return out


# ------------------------------------------------------------------ GPU arm
def main():
    a = args_()
    wl = workload(a)
    if a.workload != "c2":
        a.log_n, a.levels, a.batch = wl["log_n"], wl["levels"], wl["batch"]
        if a.alpha == 0:
            a.alpha = wl["alpha"]
    if a.impl == "reference":
        return reference_arm(a)
    if a.kernel:
        return kernel_arm(a)
    if a.serve:
        return serve_arm(a)
    if a.table3:
        return table3_arm(a)
    if a.boot:
        return boot_arm(a)
    if a.deep:
        return deep_arm(a)
    import numpy as np
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    c1_pool = c1_job = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        # the oracle's whole C1 inference runs on one host core while the
        # GPU is timed (a spawned process, started before any CUDA call)
        import multiprocessing as mp
        c1_pool = mp.get_context("spawn").Pool(1)
        c1_job = c1_pool.apply_async(c1_oracle_full)
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        from paper_2409_07751_gb300 import build
        build.build()
    if dist:
        dist.barrier()
    from paper_2409_07751_gb300 import ckks as G
    from paper_2409_07751_gb300 import workloads as W

    # a dedicated (non-default) stream shared by the library and the timing events
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    tuned = None
    if a.alpha == 0:
        a.alpha, a.p_bits, tuned = G.autotune_keyswitch(a.log_n, a.levels, a.max_qp_bits, batch=8,
                                                        device=local)
    ctx = G.Context(a.log_n, a.levels, a.alpha, p_bits=a.p_bits, device=local)
    ctx.set_stream(stream.cuda_stream)
    # CTAs per SM of each NTT kind, by measurement on this context
    ntt_chosen, ntt_ms = ctx.autotune_ntt(8)
    ntt_tune = {"chosen_ctas_per_sm": ntt_chosen,
                "ms_at_2_and_1_ctas_per_sm": {k: [round(v[0], 3), round(v[1], 3)]
                                              for k, v in ntt_ms.items()},
                "workload": "HMult, HRot, constant product, rescale, forward NTT; batch 8 "
                            "at the top level"}
    model, Xcal, X = model_and_inputs(a, rank)
    m = calibrate_for(a, G.calibrate, model, Xcal, gpu_design(G))
    gm = G.Model(ctx, m)
    gm.set_graphs(a.graphs)
    depth = sum(gm.layer_depth(i) for i in range(gm.n_layers))
    slack = a.levels - depth
    plan = shard_plan(rank, a.batch)
    if wl["uneven"]:
        levels = W.uneven_levels(a.batch, a.levels, slack, seed=plan["level_seed"])
    else:  # encrypted at the level the network needs (the chain's spare levels unused)
        levels = np.full(a.batch, min(a.levels, depth))
    keys = G.Keys(ctx, W.SEED_KEYS, gm.rotations())
    K = gm.layer_chunks(0)[0]

    def packed(rows):  # the first layer's rows of each input (K chunks of a wide input)
        return np.concatenate([np.atleast_2d(gm.pack_input(r)) for r in rows])

    cts = []
    for lv in sorted(set(int(x) for x in levels)):
        sel = np.nonzero(levels == lv)[0]
        cts.append(G.encrypt(ctx, keys, packed(X[sel]), lv, W.SEED_ENC,
                             first_index=K * (int(sel[0]) + plan["first_index"])))

    def step():
        out = G.kan_infer(ctx, keys, gm, cts)
        out.close()
        return out

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- timed region (no per-launch events: they cost time
    # between small kernels), then the same K steps again with per-launch
    # CUDA events for the per-kind durations of the roofline
    before = ctx.launch_counts()
    clk = Clocks(local)
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    ev[0].record(stream)
    for i in range(a.steps):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    after = ctx.launch_counts()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(a.steps)]
    elapsed = reduce_max(ev[0].elapsed_time(ev[-1]), dist, "cuda")
    launches = sum(after[k] - before[k] for k in after if k != "copy")
    value = world * a.batch * a.steps / (elapsed / 1000.0)
    ctx.profile(True)
    barrier()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for i in range(a.steps):
        step()
    p1.record(stream)
    torch.cuda.synchronize()
    barrier()
    profiled_ms = p0.elapsed_time(p1)
    prof = ctx.profile_collect()
    ctx.profile(False)

    # roofline of the dominant kernel kind
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    kinds = {k: v for k, v in prof.items() if k != "copy"}
    dom = max(kinds, key=lambda k: kinds[k][0])
    ms, by, n, mm = kinds[dom]
    achieved = by / (ms / 1000.0) / 1e9
    total_ms = sum(v[0] for v in kinds.values())
    traffic = None
    if dom == "modup_ntt" and MODUP_TRAFFIC_RATIO is not None:
        traffic = MODUP_TRAFFIC_RATIO * by / n
    # the fraction is taken against HBM (algorithmic bytes / launch time /
    # measured copy bandwidth); the integer roofline of the same launches is
    # reported beside it against the measured register-only butterfly rate
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    int_peaks = {"products_per_s": ctx.int_peak(0), "butterflies_per_s": ctx.int_peak(1),
                 "shoup_products_per_s": ctx.int_peak(2)}
    if mm > 0:
        alu = mm / (ms / 1000.0) / 1e9
        bpk = int_peaks["butterflies_per_s"] / 1e9
        roofline["alu"] = {"achieved": alu, "unit": "G modmul/s", "peak": bpk, "frac": alu / bpk,
                           "peak_source": "measured: register-only lazy forward butterflies "
                                          "(ckks_int_peak kind 1)",
                           "modmul_per_launch": mm / n}
    roofline.update({"algorithmic_bytes_per_launch": by / n, "avg_launch_ms": ms / n,
                     "share_of_kernel_time": ms / total_ms,
                     "kernel_ms_per_step": total_ms / a.steps,
                     "profiled_ms_per_step": profiled_ms / a.steps,
                     "copy_ms_per_step": prof.get("copy", (0.0,))[0] / a.steps})
    shares = {k: round(v[0] / total_ms, 4) for k, v in sorted(kinds.items(), key=lambda kv: -kv[1][0])}
    # per kind: ms per step, algorithmic GB/s and G modmul/s over its launches
    rates = {k: {"ms_per_step": round(v[0] / a.steps, 2),
                 "GBps": round(v[1] / (v[0] / 1000.0) / 1e9, 1) if v[0] > 0 else None,
                 "Gmodmul_per_s": round(v[3] / (v[0] / 1000.0) / 1e9, 1) if v[0] > 0 and v[3] else None,
                 "hbm_frac": round(v[1] / (v[0] / 1000.0) / 1e9 / peak, 4) if v[0] > 0 else None,
                 "alu_frac": round(v[3] / (v[0] / 1000.0) / int_peaks["butterflies_per_s"], 4)
                 if v[0] > 0 and v[3] else None}
             for k, v in sorted(kinds.items(), key=lambda kv: -kv[1][0])[:8]}

    def timed(fn, reps):
        def run():
            r = fn()
            if r is not None:
                r.close()
        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0 / reps

    # ---------------- the plain form: one request at a time, fusion off
    plain = None
    if not a.no_micro:
        one = G.encrypt(ctx, keys, packed(X[:1]), a.levels, 9, 0)
        gm.set_graphs(False)
        plain = {}
        for fused in (False, True):
            ctx.set_fusion(fused)
            s = timed(lambda: G.kan_infer(ctx, keys, gm, [one]), 2)
            plain["fused" if fused else "unfused"] = {"value": 1.0 / s, "unit": UNIT, "batch": 1}
        ctx.set_fusion(True)
        plain["fused_graphs"] = None
        gm.set_graphs(True)
        s = timed(lambda: G.kan_infer(ctx, keys, gm, [one]), 3)  # eager, capture, replays
        s = timed(lambda: G.kan_infer(ctx, keys, gm, [one]), 3)
        plain["fused_graphs"] = {"value": 1.0 / s, "unit": UNIT, "batch": 1}
        gm.set_graphs(a.graphs)
        one.close()
        plain["batched_over_plain"] = value / world / plain["unfused"]["value"]

    # ---------------- the same batch replayed from CUDA graphs (no profiling)
    graph_replay = None
    if not a.no_micro and not a.graphs:
        gm.set_graphs(True)
        step()  # eager run of each layer shape
        step()  # capture
        s = timed(lambda: G.kan_infer(ctx, keys, gm, cts), 2)
        graph_replay = {"value": world * a.batch / s, "unit": UNIT, "batch": a.batch}
        gm.set_graphs(False)

    # ---------------- micro: HMult / HRot per second at N=2^16, l in {37, 19, 2}
    micro = None
    if not a.no_micro:
        micro = {}
        for lv in (a.levels, a.levels // 2, 1):
            for B in (1, 8, 64):
                x = G.encrypt(ctx, keys, X[:B], lv, 9, 0)
                for name, fn in (("hmult", lambda: G.mul(ctx, keys, x, x)),
                                 ("hrot", lambda: G.rotate(ctx, keys, x, 1))):
                    s = timed(fn, 3 if B < 64 else 2)
                    micro["%s_per_s_l%d_b%d" % (name, lv + 1, B)] = B / s
                x.close()
        rows = 2 * (a.levels + 1) * 8
        buf = torch.zeros(rows * ctx.N, dtype=torch.int64, device="cuda")
        for inv in (False, True):
            s = timed(lambda: ctx.ntt(buf.data_ptr(), rows, a.levels + 1, inv), 5)
            micro["%s_limbs_per_s" % ("intt" if inv else "ntt")] = rows / s
        del buf

    # ---------------- seed-compressed keys: the same batched step and the
    # top-level HMult / HRot with the switching keys' uniform halves
    # regenerated before each key switch
    compressed = None
    if not a.no_micro:
        ck = G.Keys(ctx, W.SEED_KEYS, gm.rotations(), public_seed=W.SEED_KEYS + 0x5EED)
        full_bytes = ck.nbytes()
        ck.compress()
        compressed = {"key_bytes_full": full_bytes, "key_bytes_compressed": ck.nbytes()}
        s = timed(lambda: G.kan_infer(ctx, ck, gm, cts), 2)
        compressed["inferences_per_s"] = world * a.batch / s
        compressed["over_full_keys"] = compressed["inferences_per_s"] / value
        for B in (1, 64):
            x = G.encrypt(ctx, ck, X[:B], a.levels, 9, 0)
            for name, fn in (("hmult", lambda: G.mul(ctx, ck, x, x)),
                             ("hrot", lambda: G.rotate(ctx, ck, x, 1))):
                compressed["%s_per_s_l%d_b%d" % (name, a.levels + 1, B)] = B / timed(fn, 3 if B < 64 else 2)
            x.close()
        ck.close()

    # ---------------- end to end through the C ABI with pinned host buffers
    e2e = None
    if not a.no_e2e:
        hin = []
        for c in cts:
            buf = torch.empty(c.words(), dtype=torch.int64, pin_memory=True)
            c.export_to(buf.data_ptr(), c.words())
            hin.append((buf, c.batch, c.level, c.scale))
        probe = G.kan_infer(ctx, keys, gm, cts)
        out_words = probe.words()
        probe.close()
        hout = torch.empty(out_words, dtype=torch.int64, pin_memory=True)
        h2d = sum(b.numel() * 8 for b, _, _, _ in hin)

        def e2e_step():
            ins = [G.Ciphertext.import_from(ctx, b.data_ptr(), B, lv, sc) for b, B, lv, sc in hin]
            out = G.kan_infer(ctx, keys, gm, ins)
            out.export_to(hout.data_ptr(), out_words)
            for c in ins:
                c.close()
            out.close()

        e2e_step()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        el_serial = reduce_max(e0.elapsed_time(e1), dist, "cuda")
        # pipelined: the next batch's inputs are copied on a second stream
        # while the current batch computes (the library's stream waits for
        # each copy through an event); every copy is inside the timed region
        cstream = torch.cuda.Stream()

        def imports():
            return [G.Ciphertext.import_from_async(ctx, b.data_ptr(), B, lv, sc, cstream.cuda_stream)
                    for b, B, lv, sc in hin]

        barrier()
        e0.record(stream)
        cstream.wait_event(e0)
        nxt = imports()
        for i in range(a.steps):
            ins = nxt
            out = G.kan_infer(ctx, keys, gm, ins)
            nxt = imports() if i + 1 < a.steps else None
            out.export_to(hout.data_ptr(), out_words)
            for c in ins:
                c.close()
            out.close()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        el = reduce_max(e0.elapsed_time(e1), dist, "cuda")
        # the host-to-device part alone: the step's inputs imported on the
        # copy stream, timed with CUDA events on it (after one untimed import,
        # so the pool's memory is mapped)
        for b, B, lv, sc in hin:
            G.Ciphertext.import_from_async(ctx, b.data_ptr(), B, lv, sc, cstream.cuda_stream).close()
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(cstream)
        held = [G.Ciphertext.import_from_async(ctx, b.data_ptr(), B, lv, sc, cstream.cuda_stream)
                for b, B, lv, sc in hin]
        h1.record(cstream)
        torch.cuda.synchronize()
        h2d_ms = h0.elapsed_time(h1)
        for c_ in held:
            c_.close()
        e2e = {"value": world * a.batch * a.steps / (el / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": out_words * 8,
               "h2d_ms_per_step": h2d_ms, "h2d_GBps": h2d / (h2d_ms / 1000.0) / 1e9,
               "serial_value": world * a.batch * a.steps / (el_serial / 1000.0),
               "path": "ckks_ct_import_async on a copy stream (next batch overlapped with the "
                       "current one) -> kan_infer -> ckks_ct_export"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": elapsed / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": config(a),
            "latency_ms": {"p50": statistics.median(step_ms),
                           "p99": float(np.percentile(step_ms, 99)), "per": "batch of %d" % a.batch},
            "roofline": roofline, "kernel_time_shares": shares, "kernel_rates": rates,
            "compressed_keys": compressed,
            "gpu_launches": launches,
            "clocks": clocks, "e2e": e2e, "plain_form": plain, "graph_replay": graph_replay,
            "keyswitch_autotune_ms": tuned, "ntt_autotune": ntt_tune, "micro": micro,
            "int_peaks": int_peaks, "depth": depth,
            "slack": slack}
    if rank == 0 and world == 1 and not a.no_extras and a.workload == "c2":
        line["configs"] = extras(local)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        from oracle import calibrate as OC
        mo = calibrate_for(a, OC.calibrate, model, Xcal, oracle_design)
        v1, sample1, _ = oracle_sample(mo, a, a.cpu_budget)
        v, sample, procs = oracle_all_cores(mo, a, a.cpu_budget)
        c1 = None
        try:
            c1_s = c1_job.get(timeout=900)
            c1 = {"value": 1.0 / c1_s, "unit": UNIT, "seconds": c1_s, "cores": 1,
                  "sample": "full inference: one whole encrypted [2,5,1] inference (N=2^15, 18 "
                            "levels), single thread, run while the GPU was timed"}
        except Exception as e:  # reported, not hidden
            c1 = {"error": repr(e)}
        c1_pool.terminate()
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
                                "sample": "%d processes, each: %s" % (procs, sample),
                                "single_thread": {"value": v1, "cores": 1, "sample": sample1},
                                "c1_full_inference": c1}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
