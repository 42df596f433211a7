"""Throughput of the Hawkes log-likelihood + gradient on one GB300.

A step is one pass of the evaluation an MCMC iteration makes: the
cut-posterior location resample (Sec. 2.2) followed by the full FP32
log-likelihood and six-component gradient (eq. 4) over all N(N-1)/2
unordered event pairs, on the N = 1,000,000 synthetic Voronoi-county
workload (3,143 counties on a 4,500 x 2,800 km box, lognormal densities,
Hawkes-burst times over 1,200 days).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  ``value`` is unordered pairs per second over all ranks
(each rank runs its own chain replica: weak scaling, no collective on the
data path).  ``--impl reference`` times the FP64 CPU oracle on a bounded
sample of the same workload instead.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "loglik+grad pairs/s at N=1M (1 and 30-chain batch); HMC ESS/s surrogate vs exact"
UNIT = "pairs/s"
WORKLOAD = "c3: N=1,000,000 events, 1,200 d, 3,143 Voronoi counties (4,500x2,800 km), resample + FP32 loglik + 6-dim grad per step"
# Algorithmic FP32 pipe operations per unordered pair (one lane op each:
# FADD, FMUL or FFMA): time difference 1, dx and dy 2, r^2 2, dt^2 1,
# background exponent 1, row and column background moments 3 + 3, beta r^2 1,
# excitation exponent 2, excitation moments 3.  The two-word coordinate split
# (4 more) is overhead, not counted.
ALG_FP32_OPS_PER_PAIR = 19
# The same count as first estimated before the kernel existed: 5 for the
# differences and r^2, 1 for dt^2, 4 for both exponent arguments, 7 for the row
# moments, 3 for the column moments and about 4 for per-pair scaling and
# selection.  The kernel needs none of those 4 (scales and masks are applied
# per row or per tile, outside the pair loop) and forms the excitation
# argument with one FMA, so 19 is the stricter count; both are reported.
ESTIMATED_FP32_OPS_PER_PAIR = 24
# log-likelihood only: the row moments SBr, SBt, SEt, SEq and the column
# moments SBr, SBt are not formed (6 fewer)
LL_FP32_OPS_PER_PAIR = 13
FP32_LANES_PER_SM = 128


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"sm_max_mhz": 2070.0}, "fallback"


def source_hash():
    h = hashlib.sha256()
    for f in ("sweep_kernel.cuh", "sweep.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2407_11349_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """Per-launch DRAM bytes of the sweep from the committed ncu summary, if it
    was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "sweep_f32_c3.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    want = source_hash()
    val, src = None, None
    for line in txt.splitlines():
        if line.startswith("traffic_bytes_per_launch:"):
            val = float(line.split(":", 1)[1].split()[0])
        if line.startswith("kernel_source_hash:"):
            src = line.split(":", 1)[1].strip()
    return val if (val is not None and src == want) else None


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def bench_batch(ds_c3, steps, warmup):
    """30 chains (N = 250,000 each, own parameters and resample stream) plus 16
    regional subsets (N = 5,000 ... 200,000) in one persistent sweep launch,
    captured in a CUDA graph, against the same 46 problems as sequential
    per-problem calls.  Returns a dict for the JSON line."""
    import torch
    from paper_2407_11349_gb300 import synth
    from paper_2407_11349_gb300.hawkes import HAWKES_F32, Batch, Hawkes

    base = synth.config_dataset("c4")
    regions = synth.regional_subsets(ds_c3, synth.regional_sizes(), seed=3)
    dss = [base] * 30 + regions
    P = len(dss)
    params = synth.chain_params(P, seed=3)
    seeds, streams = [3] * P, list(range(P))
    pairs = sum(d.n * (d.n - 1) / 2 for d in dss)
    stream = torch.cuda.current_stream()  # the dedicated stream main() made current
    hks = [Hawkes(torch.cuda.current_device(), stream.cuda_stream).load(d) for d in dss]
    dp = torch.tensor(params, dtype=torch.float64, device="cuda")
    dout = torch.zeros((P, 7), dtype=torch.float64, device="cuda")
    b = Batch(hks, seeds, streams, HAWKES_F32, stream.cuda_stream)
    variant, chunk, order, tune_ms = b.tune(dp.data_ptr(), dout.data_ptr(), reps=1)
    kc, n_groups = b.config()[3:]
    b.capture(dp.data_ptr(), dout.data_ptr())
    ev = lambda: torch.cuda.Event(enable_timing=True)
    douts = torch.zeros((P, 7), dtype=torch.float64, device="cuda")

    def batched(it):
        e0, e1 = ev(), ev()
        e0.record(stream)
        b.run(dp.data_ptr(), it, dout.data_ptr())
        e1.record(stream)
        b.wait()
        return e0.elapsed_time(e1)

    def sequential(it):  # the same work as one call per problem (async entry point, same stream)
        e0, e1 = ev(), ev()
        e0.record(stream)
        for p in range(P):
            hks[p].resample(seeds[p], streams[p], it)
            hks[p].loglik_grad_async(dp[p].data_ptr(), douts[p].data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    for k in range(warmup):
        batched(k)
        sequential(k)
    # alternate the two so that drift of the clock or the L2 state hits both
    tb, ts = [], []
    for k in range(steps):
        tb.append(batched(100 + k))
        ts.append(sequential(100 + k))
    batch_out, seq_last = dout.cpu().numpy(), douts.cpu().numpy()
    agree = float(np.max(np.abs(seq_last[:, 0] - batch_out[:, 0]) / np.abs(seq_last[:, 0])))
    # the same batch with one chain per CTA (the tuned k = 1 configuration)
    t1 = []
    if kc > 1:
        b.set_chains_per_cta(1)
        b.capture(dp.data_ptr(), dout.data_ptr())
        batched(200)
        t1 = [batched(201 + k) for k in range(3)]
    b.close()
    for h in hks:
        h.close()
    ratios = sorted(s_ / b_ for s_, b_ in zip(ts, tb))
    mb, ms_ = statistics.median(tb), statistics.median(ts)
    return {"value": pairs / (mb / 1000.0), "unit": UNIT, "sequential_value": pairs / (ms_ / 1000.0),
            "speedup_vs_sequential": ms_ / mb, "speedup_per_repeat": [round(r, 4) for r in ratios],
            "speedup_min": ratios[0], "speedup_max": ratios[-1], "repeats": steps,
            "ms_per_step": mb, "ms_per_step_all": [round(v, 2) for v in tb],
            "sequential_ms_per_step": ms_, "sequential_ms_all": [round(v, 2) for v in ts],
            "problems": P, "pairs_per_step": pairs,
            "tuned": {"variant": variant, "chunk_tiles": chunk, "order": order, "sweep_ms": tune_ms,
                      "chains_per_cta": kc, "groups": n_groups},
            "one_chain_per_cta_ms_per_step": statistics.median(t1) if t1 else None,
            "graph": True, "loglik_rel_diff_batch_vs_sequential": agree,
            "config": "30 chains x N=250,000 (own params, own resample stream) + 16 regional subsets "
                      "N=5,000..200,000 (sum 899,416); one persistent launch per kernel family in a "
                      "CUDA graph (chains sharing their times swept chains_per_cta at a time); "
                      "medians of alternating batched / sequential repeats"}


def bench_batch_kc(workload, kcs, chunk=64, repeats=3):
    """Whole batched steps (CUDA graph) at fixed chains per CTA: "c4" is the
    30-chain batch of the benchmark (30 x N = 250,000 plus the 16 regional
    subsets), "c2x4" four chains of the N = 100,000 workload (a small case
    for profiling).  Sweep variant 0, item order 0, the given chunk length.
    Returns {chains_per_cta: median ms per step}."""
    import torch
    from paper_2407_11349_gb300 import synth
    from paper_2407_11349_gb300.hawkes import HAWKES_F32, Batch, Hawkes

    if workload == "c4":
        dss = [synth.config_dataset("c4")] * 30 + synth.regional_subsets(
            synth.config_dataset("c3"), synth.regional_sizes(), seed=3)
    else:
        dss = [synth.config_dataset("c2")] * 4
    P = len(dss)
    stream = torch.cuda.current_stream()
    hks = [Hawkes(torch.cuda.current_device(), stream.cuda_stream).load(d) for d in dss]
    dp = torch.tensor(synth.chain_params(P, seed=3), dtype=torch.float64, device="cuda")
    dout = torch.zeros((P, 7), dtype=torch.float64, device="cuda")
    b = Batch(hks, [3] * P, list(range(P)), HAWKES_F32, stream.cuda_stream)
    out = {}
    for kc in kcs:
        b.set_config(0, chunk, 0)
        b.set_chains_per_cta(kc)
        b.capture(dp.data_ptr(), dout.data_ptr())
        ts = []
        for k in range(repeats + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run(dp.data_ptr(), k, dout.data_ptr())
            e1.record(stream)
            b.wait()
            if k:
                ts.append(e0.elapsed_time(e1))
        out[kc] = statistics.median(ts)
    b.close()
    for h in hks:
        h.close()
    return out


def bench_hmc(n_events, cut=True, chains=4, leapfrog=10, warmup=300, draws=300, ref_rounds=0,
              lite=False, flags=0, moves=0, train_from="last", progress=None, checkpoint=None,
              resume=None):
    """Min bulk ESS per second of exact HMC vs surrogate HMC, same data, same
    adapted step size and metric.  cut=True: locations resampled every
    iteration (the cut-posterior scheme); cut=False: locations held fixed,
    so both samplers target p(Theta | X, t) exactly and their posterior
    means must agree within Monte Carlo error.  The surrogate is trained on
    the exact evaluations of the exact-HMC warmup from its last slow
    adaptation window on.  Unless lite, three more samplers run from the
    same start: the anchored surrogate, three surrogate moves per location
    draw, and the paper's univariate Metropolis-Hastings.  ref_rounds > 0
    (cut only): every sampler is also compared with an independent sample
    of the cut posterior.  flags: extra likelihood flags (e.g. the exact
    underflow skip, which changes no result).  moves > 1 (lite runs): the
    plain and (cut) feature surrogates also run with that many moves per
    location draw.  train_from: "last" trains the network on the warmup's
    evaluations from its last slow adaptation window on, "fast" on every
    evaluation after the first fast window (15% of the warmup).  progress:
    a file that receives each finished part as one JSON line.  checkpoint:
    write the warmup's end state (chains, step sizes, metric, iteration,
    sampler RNG) and the training sets to this file and return; resume:
    start from such a file instead of running the warmup (a long run split
    over two processes)."""
    import pickle
    from paper_2407_11349_gb300 import diagnostics as dg
    from paper_2407_11349_gb300 import hmc, synth
    from paper_2407_11349_gb300.hawkes import MLP

    # events with the model's space-time structure on a 40 x 40 grid of 50 km
    # counties over 1,200 days (drawn from the model itself, so the posterior
    # is concentrated near the generating parameters)
    ds = synth.clustered_dataset(n_events, T=1200.0, nx=40, ny=40, seed=4)
    eta0 = np.log(synth.DEFAULT_PARAMS)
    prior = hmc.Prior(eta0)
    tgt = hmc.HawkesTarget(ds, chains, seed=4, flags=flags)
    init = np.tile(eta0, (chains, 1)) + np.random.default_rng(4).normal(0, 0.01, (chains, 6))
    ex = hmc.Sampler(tgt, prior, init, n_leapfrog=leapfrog, seed=1, cut=cut)
    ex.record = []
    # under the cut scheme the warmup also records each location draw's
    # feature: the exact log-likelihood at a fixed anchor (the starting
    # point) under that draw, the seventh input of the feature network
    a_f = eta0.copy() if cut else None
    if resume:
        with open(resume, "rb") as f:
            ck = pickle.load(f)
        ex.set_state(ck["state"])
        ex.record = None
        t_warm, n_warm_exact = ck["t_warm"], ck["n_warm_exact"]
        X, Y, feat = ck["X"], ck["Y"], ck["feat"]
    else:
        t0 = time.perf_counter()
        last = ex.warmup(warmup, feature_anchor=a_f)
        t_warm = time.perf_counter() - t0
        n_warm_exact = tgt.n_exact
        first = last if train_from == "last" else int(0.15 * warmup)
        rec = ex.record[1 + first * (leapfrog + 1):]
        X, Y = hmc.training_set(rec)
        feat = hmc.training_set(rec, with_feature=True) if cut else None
        ex.record = None
        if checkpoint:
            with open(checkpoint, "wb") as f:
                pickle.dump({"state": ex.state(), "t_warm": t_warm, "n_warm_exact": n_warm_exact,
                             "X": X, "Y": Y, "feat": feat}, f)
            tgt.close()
            return {"checkpoint": checkpoint, "warmup_s": t_warm, "warmup_exact_evals": n_warm_exact,
                    "training_pairs": int(X.shape[0])}
    net = MLP(torch_device(), seed=2)
    t0 = time.perf_counter()
    net.set_data(X, Y)
    loss = net.train(4000, batch=512, lr=1e-3, seed=3)
    t_train = time.perf_counter() - t0
    q_start, eps, cov = ex.q.copy(), ex.eps.copy(), ex.cov.copy()
    field = hmc.SurrogateField(net, chains)
    net_f = field_f = None
    if cut:
        Xf, Yf, Ff = feat
        net_f = MLP(torch_device(), seed=2)
        net_f.set_data(Xf, Yf, Ff)
        loss_f = net_f.train(4000, batch=512, lr=1e-3, seed=3)
        field_f = hmc.SurrogateField(net_f, chains, feature=True)

    def note(part, val):
        if progress:
            with open(progress, "a") as f:
                f.write(json.dumps({part: val}, default=float) + "\n")

    note("warmup", {"seconds": t_warm, "exact_evals": n_warm_exact, "training_pairs": int(X.shape[0]),
                    "train_loss": loss, "train_s": t_train})

    def run(name, sampler, **kw):
        n0 = tgt.n_exact
        d, acc, sec = sampler.sample(draws, **kw)
        summ = dg.summary(d, hmc.NAMES)
        ess = min(v["bulk_ess"] for v in summ.values())
        r = {"min_bulk_ess": ess, "seconds": sec, "ess_per_s": ess / sec,
             "accept": float(acc.mean()), "exact_evals": tgt.n_exact - n0,
             "exact_evals_per_ess": (tgt.n_exact - n0) / max(ess, 1e-9),
             "mean": {k: summ[k]["mean"] for k in hmc.NAMES}, "mcse": {k: summ[k]["mcse"] for k in hmc.NAMES}}
        note(name, r)
        return summ, r

    def hmc_sampler(seed):
        smp = hmc.Sampler(tgt, prior, q_start, n_leapfrog=leapfrog, seed=seed, cut=cut)
        smp.eps, smp.iteration = eps, ex.iteration
        smp.set_cov(cov)
        return smp

    summaries, res = {}, {}
    summaries["exact"], res["exact"] = run("exact", ex)
    summaries["surrogate"], res["surrogate"] = run("surrogate", hmc_sampler(5), field=field)
    if cut:
        # the network told about each draw through its seventh input
        summaries["surrogate_feature"], res["surrogate_feature"] = run("surrogate_feature", hmc_sampler(9), field=field_f,
                                                                       feature_anchor=a_f)
        res["surrogate_feature"]["train_loss"] = loss_f
    if lite and moves > 1:
        # several surrogate moves per location draw (1 + moves exact
        # evaluations; the feature network adds the anchor's evaluation)
        nm = f"surrogate_{moves}_moves"
        summaries[nm], res[nm] = run(nm, hmc_sampler(8), field=field, moves=moves)
        if cut:
            nm = f"surrogate_feature_{moves}_moves"
            summaries[nm], res[nm] = run(nm, hmc_sampler(10), field=field_f, feature_anchor=a_f,
                                         moves=moves)
    if not lite:
        # the anchored surrogate: each iteration's field is shifted by the
        # exact minus the network's gradient at a fixed anchor (the median of
        # the training points) under that iteration's locations
        summaries["surrogate_anchored"], res["surrogate_anchored"] = run(
            "surrogate_anchored", hmc_sampler(7), field=field, anchor=np.median(X, axis=0))
        # three surrogate moves per location draw (1 + 3 exact evaluations)
        summaries["surrogate_3_moves"], res["surrogate_3_moves"] = run("surrogate_3_moves", hmc_sampler(8), field=field,
                                                                       moves=3)
        # the paper's sampler: univariate Metropolis-Hastings, same target and start
        mh = hmc.MHSampler(tgt, prior, q_start, seed=6, cut=cut)
        mh.iteration = ex.iteration
        mh.log_scale = np.log(np.sqrt(np.stack([np.diag(c) for c in cov]))) + np.log(2.38 / np.sqrt(6.0))
        mh.warmup(50)
        summaries["univariate_mh"], res["univariate_mh"] = run("univariate_mh", mh)
    s_ex = summaries["exact"]
    for k, summ in summaries.items():
        res[k]["ess_per_s_vs_exact"] = res[k]["ess_per_s"] / res["exact"]["ess_per_s"]
        if k != "exact":
            res[k]["mean_diff_vs_exact_in_mcse_units"] = {
                nm: float(abs(s_ex[nm]["mean"] - summ[nm]["mean"]) / np.hypot(s_ex[nm]["mcse"], summ[nm]["mcse"]))
                for nm in hmc.NAMES}
    ref = None
    if cut and ref_rounds > 0:
        # the cut posterior itself: exact HMC with each location draw held
        # fixed, pooled over ref_rounds x chains draws of X
        t0 = time.perf_counter()
        d_ref = hmc.cut_posterior_reference(tgt, prior, q_start, cov, eps, ref_rounds, burn=30, draws=100,
                                            n_leapfrog=leapfrog, seed=11)
        m_cr = d_ref.mean(axis=1)  # one mean per (chain, round)
        ref_mean = m_cr.mean(axis=0)
        ref_se = m_cr.std(axis=0, ddof=1) / np.sqrt(m_cr.shape[0])
        ref = {"location_draws": int(m_cr.shape[0]), "draws_per_location": int(d_ref.shape[1]),
               "seconds": time.perf_counter() - t0,
               "mean": {k: float(ref_mean[i]) for i, k in enumerate(hmc.NAMES)},
               "se": {k: float(ref_se[i]) for i, k in enumerate(hmc.NAMES)},
               "diff_in_se_units": {nm: {k: float(abs(sm[k]["mean"] - ref_mean[i]) / np.hypot(sm[k]["mcse"],
                                                                                             ref_se[i]))
                                         for i, k in enumerate(hmc.NAMES)}
                                    for nm, sm in summaries.items() if nm != "univariate_mh"}}
    net.close()
    if net_f is not None:
        net_f.close()
    tgt.close()
    note("cut_posterior_reference", ref)
    out = {"n_events": ds.n, "chains": chains, "leapfrog": leapfrog, "warmup_iters": warmup,
           "draws_per_chain": draws, "training_pairs": int(X.shape[0]), "train_loss": loss,
           "warmup_exact_evals": n_warm_exact, "train_from": train_from,
           **res,
           "speedup_ess_per_s": res["surrogate"]["ess_per_s_vs_exact"],
           # at large N, where the exact evaluations dominate the time, the
           # ratio of exact evaluations per effective sample is the ESS/s ratio
           "speedup_when_exact_evaluations_dominate": (res["exact"]["exact_evals_per_ess"] /
                                                       res["surrogate"]["exact_evals_per_ess"]),
           "warmup_s": t_warm, "train_s": t_train,
           "cut_posterior_reference": ref,
           "locations": "resampled every iteration (cut posterior)" if cut else "fixed",
           "note": "all samplers share the exact-HMC warmup's step size and dense metric; the surrogate "
                   "is trained on the warmup's exact evaluations; data: clustered synthetic events on a "
                   "40x40 grid of 50 km counties over 1,200 days"}
    return out


def bench_mh(n_events, chains=30, warmup=150, draws=400, flags=0, seed=4):
    """The paper's sampler at its chain count (Sec. 2.2, 3.2): univariate
    random-walk Metropolis-Hastings on log-parameters under the cut scheme,
    all chains in lockstep, each update one batched log-likelihood-only
    evaluation of every chain.  Reports the worst parameter's bulk and tail
    ESS and R-hat, as the paper's Sec. 3.2 does, and the time."""
    from paper_2407_11349_gb300 import diagnostics as dg
    from paper_2407_11349_gb300 import hmc, synth
    ds = synth.clustered_dataset(n_events, T=1200.0, nx=40, ny=40, seed=seed)
    eta0 = np.log(synth.DEFAULT_PARAMS)
    prior = hmc.Prior(eta0)
    tgt = hmc.HawkesTarget(ds, chains, seed=seed, flags=flags)
    init = np.tile(eta0, (chains, 1)) + np.random.default_rng(seed).normal(0, 0.01, (chains, 6))
    mh = hmc.MHSampler(tgt, prior, init, seed=6, cut=True)
    t0 = time.perf_counter()
    mh.warmup(warmup)
    t_warm = time.perf_counter() - t0
    n0 = tgt.n_exact
    d, acc, sec = mh.sample(draws)
    summ = dg.summary(d, hmc.NAMES)
    worst = min(hmc.NAMES, key=lambda k: summ[k]["bulk_ess"])
    out = {"n_events": ds.n, "chains": chains, "warmup_iters": warmup, "draws_per_chain": draws,
           "seconds_warmup": t_warm, "seconds_sampling": sec, "accept": float(acc.mean()),
           "evaluations": tgt.n_exact - n0, "evaluations_per_s": (tgt.n_exact - n0) / sec,
           "worst_parameter": worst, "worst_bulk_ess": summ[worst]["bulk_ess"],
           "worst_tail_ess": min(v["tail_ess"] for v in summ.values()),
           "max_rhat": max(v["rhat"] for v in summ.values()),
           "min_bulk_ess_per_s": summ[worst]["bulk_ess"] / sec,
           "summary": summ,
           "note": "log-likelihood-only batched evaluations (HAWKES_LOGLIK_ONLY); clustered synthetic "
                   "events on a 40x40 grid of 50 km counties over 1,200 days"}
    tgt.close()
    return out


def accuracy_c3(hk, ds, p):
    """The FP32 path's seven outputs on the c3 workload after resample(2, 0, 0)
    against the oracle's values stored in tests/golden/oracle_c3.json (written
    from the oracle alone), once the inputs are checked to be the same:
    relative error of each output against itself, and against
    max(|g_k|, 1e-3 sum_i |d ell_i / d p_k|) (the floor the parity tests use
    for components that cancel)."""
    from paper_2407_11349_gb300 import synth
    path = os.path.join(ROOT, "tests", "golden", "oracle_c3.json")
    if not os.path.exists(path):
        return {"against": None, "note": "tests/golden/oracle_c3.json missing"}
    doc = json.load(open(path))
    hk.resample(2, 0, 0)
    x, y = hk.locations()
    if not synth.same_inputs(synth.fingerprint({"t": ds.t, "x": x, "y": y, "s": ds.s})["stats"],
                             doc["inputs"]["stats"]):
        return {"against": None, "note": "c3 inputs differ from the stored oracle's"}
    ll, g = hk.loglik_grad(p, 0)
    got = np.concatenate([[ll], g])
    ref = np.asarray(doc["loglik_grad"])
    raw = np.abs(got - ref) / np.abs(ref)
    floor = np.maximum(np.abs(ref), 1e-3 * np.asarray(doc["abs_row_sums"]))
    names = ["loglik", "d_mu", "d_tau_x", "d_tau_t", "d_theta", "d_omega", "d_h"]
    return {"against": "FP64 oracle totals, tests/golden/oracle_c3.json (inputs fingerprint-matched)",
            "rel_err": {k: float(v) for k, v in zip(names, raw)},
            "rel_err_floored": {k: float(v) for k, v in zip(names, np.abs(got - ref) / floor)},
            "targets": {"loglik": 1e-6, "grad": 1e-5}}


def torch_device():
    import torch
    return torch.cuda.current_device()


def cpu_baseline(ds, seconds=15.0):
    """The FP64 oracle on the host cores, on a bounded contiguous row window in
    the middle of the workload (every row against all N sources)."""
    import oracle
    threads = oracle.max_threads()
    n = ds.n
    x, y, s = ds.x, ds.y, ds.s
    p = ds.params
    mid = n // 2
    m = 4 * threads
    while True:  # grow the window until it takes about `seconds`
        m = min(m, n - mid)
        t0 = time.perf_counter()
        oracle.loglik_grad(ds.t, x, y, p, s=s, row_begin=mid, row_end=mid + m, threads=threads)
        dt = time.perf_counter() - t0
        if dt >= 0.6 * seconds or m >= n - mid:
            break
        m = int(m * min(8.0, 1.1 * seconds / max(dt, 1e-3)))
    # m rows x (n - 1) sources = m (n - 1) / 2 unordered-pair equivalents of the full sum
    value = m * (n - 1) / 2 / dt
    return {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"rows [{mid}, {mid + m}) of the N={n} workload, each against all sources "
                      f"({m * (n - 1):.3g} ordered pairs in {dt:.1f} s); scaled as m(N-1)/2 pairs"}


def run_reference(args):
    """--impl reference: the CPU oracle timed on bounded samples of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2407_11349_gb300 import synth
    import oracle
    ds = synth.config_dataset("c3")
    threads = oracle.max_threads()
    n, mid = ds.n, ds.n // 2
    # size each step so the whole run stays within a few minutes
    budget = 150.0 / max(args.steps + args.warmup, 1)
    m = 4 * threads
    while True:
        m = min(m, n - mid)
        t0 = time.perf_counter()
        oracle.loglik_grad(ds.t, ds.x, ds.y, ds.params, s=ds.s, row_begin=mid, row_end=mid + m,
                           threads=threads)
        dt = time.perf_counter() - t0
        if dt >= 0.6 * budget or m >= n - mid:
            break
        m = int(m * min(8.0, 1.1 * budget / max(dt, 1e-3)))
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.loglik_grad(ds.t, ds.x, ds.y, ds.params, s=ds.s, row_begin=mid, row_end=mid + m,
                           threads=threads)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    T = sum(times)
    value = args.steps * m * (n - 1) / 2 / T
    sample = (f"per step rows [{mid}, {mid + m}) of the N={n} workload against all sources, "
              f"scaled as m(N-1)/2 pairs")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "oracle_sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 30-chain batch measurement")
    ap.add_argument("--batch-only", default=None, choices=["c4", "c2x4"],
                    help="time only batched steps at the chains-per-CTA values of --batch-kc")
    ap.add_argument("--batch-kc", default="1,2,4", help="with --batch-only: chains per CTA to time")
    ap.add_argument("--batch-chunk", type=int, default=64, help="with --batch-only: chunk length")
    ap.add_argument("--hmc-cut-reference", type=int, default=6,
                    help="location draws per chain for the independent cut-posterior reference (0: off)")
    ap.add_argument("--hmc-only", action="store_true",
                    help="run only the HMC comparison (cut scheme, exact vs surrogate) and print it")
    ap.add_argument("--hmc-fixed", action="store_true",
                    help="with --hmc-only: locations held fixed instead of the cut scheme")
    ap.add_argument("--hmc-spatial", action="store_true",
                    help="with --hmc-only: exact evaluations with the spatial skip (chain by chain)")
    ap.add_argument("--mh-only", action="store_true",
                    help="run only the paper's univariate MH sampler (30 chains, log-likelihood only)")
    ap.add_argument("--mh-n", type=int, default=100_000)
    ap.add_argument("--mh-chains", type=int, default=30)
    ap.add_argument("--mh-warmup", type=int, default=150)
    ap.add_argument("--mh-draws", type=int, default=400)
    ap.add_argument("--hmc-ref-rounds", type=int, default=0,
                    help="with --hmc-only: location draws per chain of the cut-posterior reference")
    ap.add_argument("--hmc-moves", type=int, default=0,
                    help="with --hmc-only: also run the surrogates with this many moves per location draw")
    ap.add_argument("--hmc-train-from", default="last", choices=["last", "fast"],
                    help="with --hmc-only: train on the warmup from its last slow window (last) or after "
                         "its first fast window (fast)")
    ap.add_argument("--hmc-progress", default=None,
                    help="with --hmc-only: append each finished part to this file as a JSON line")
    ap.add_argument("--hmc-checkpoint", default=None,
                    help="with --hmc-only: save the warmup's end state and training sets here and stop")
    ap.add_argument("--hmc-resume", default=None,
                    help="with --hmc-only: start from a --hmc-checkpoint file instead of warming up")
    ap.add_argument("--hmc-chains", type=int, default=4)
    ap.add_argument("--hmc-warmup", type=int, default=300)
    ap.add_argument("--hmc-draws", type=int, default=300)
    ap.add_argument("--hmc-n", type=int, default=50_000,
                    help="events for the HMC ESS/s comparison (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--batch-repeats", type=int, default=7,
                    help="alternating batched / sequential repeats of the 30-chain batch")
    ap.add_argument("--variant", type=int, default=-1,
                    help="sweep kernel variant (default: autotuned)")
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3"],
                    help="c3 (default) is the benchmark; c1/c2 are smaller cases for profiling")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_2407_11349_gb300 import synth
    from paper_2407_11349_gb300.hawkes import (HAWKES_BG_TIME, HAWKES_F32, HAWKES_LOGLIK_ONLY,
                                               HAWKES_SKIP_SPATIAL, HAWKES_SKIP_UNDERFLOW, Hawkes)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.batch_only:
        torch.cuda.set_stream(torch.cuda.Stream())
        r = bench_batch_kc(args.batch_only, [int(k) for k in args.batch_kc.split(",")], args.batch_chunk)
        print(json.dumps({"batch_only": args.batch_only, "chunk": args.batch_chunk,
                          "ms_per_step_by_chains_per_cta": r}))
        return
    if args.mh_only:
        torch.cuda.set_stream(torch.cuda.Stream())
        r = bench_mh(args.mh_n, chains=args.mh_chains, warmup=args.mh_warmup, draws=args.mh_draws,
                     flags=HAWKES_SKIP_UNDERFLOW)
        print(json.dumps({"mh_only": r}))
        return
    if args.hmc_only:
        # one HMC comparison at a chosen size (exact vs surrogate; an exact
        # skip of zero terms on: same results, less work)
        torch.cuda.set_stream(torch.cuda.Stream())
        r = bench_hmc(args.hmc_n, cut=not args.hmc_fixed, chains=args.hmc_chains, warmup=args.hmc_warmup,
                      draws=args.hmc_draws, lite=True, ref_rounds=args.hmc_ref_rounds,
                      moves=args.hmc_moves, train_from=args.hmc_train_from, progress=args.hmc_progress,
                      checkpoint=args.hmc_checkpoint, resume=args.hmc_resume,
                      flags=HAWKES_SKIP_SPATIAL if args.hmc_spatial else HAWKES_SKIP_UNDERFLOW)
        print(json.dumps({"hmc_only": r}))
        return
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    # one dedicated stream for the library, the L2 flush and the timing events
    torch.cuda.set_stream(torch.cuda.Stream())

    ds = synth.config_dataset(args.workload)
    n = ds.n
    pairs = n * (n - 1) / 2
    stream = torch.cuda.current_stream()
    assert stream.cuda_stream != 0
    hk = Hawkes(local, stream.cuda_stream)
    hk.load(ds)
    p = ds.params
    chain = rank  # each rank is an independent chain replica
    hk.resample(2, chain, 0)
    if args.variant >= 0:
        hk.set_variant(args.variant)
        variant, tune_ms = args.variant, []
    else:
        variant, tune_ms = hk.tune(p, reps=1)  # autotuner: fastest sweep variant for this N

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def step(k):
        hk.resample(2, chain, k)
        return hk.loglik_grad(p, HAWKES_F32)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    hk.profile(True)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            ll, g = step(args.warmup + k)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    prof = hk.profile(False)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    T = sum(step_ms) / 1000.0
    if world > 1:
        t = torch.tensor([T], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        T = float(t.item())
    value = world * args.steps * pairs / T

    sweep_launches, sweep_ms = prof["sweep"]
    sweep_avg_s = sweep_ms / max(sweep_launches, 1) / 1000.0
    pk, pk_src = peaks()
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak_ops = sms * FP32_LANES_PER_SM * sm_mhz * 1e6
    achieved_ops = ALG_FP32_OPS_PER_PAIR * pairs / sweep_avg_s
    launches = sum(v[0] for v in prof.values())

    # the same step with the exact-underflow tile skip (reported separately):
    # identical result, less work
    skip_ms = []
    for k in range(args.steps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        hk.resample(2, chain, 500 + k)
        ll_s, g_s = hk.loglik_grad(p, HAWKES_F32 | HAWKES_SKIP_UNDERFLOW)
        e1.record(stream)
        torch.cuda.synchronize()
        if k:
            skip_ms.append(e0.elapsed_time(e1))
    hk.resample(2, chain, 500 + args.steps)
    ll_f, g_f = hk.loglik_grad(p, HAWKES_F32)
    skip = {"ms_per_step": sum(skip_ms) / len(skip_ms),
            "pairs_per_s_equivalent": pairs / (sum(skip_ms) / len(skip_ms) / 1000.0),
            "speedup": (1000 * T / args.steps) / (sum(skip_ms) / len(skip_ms)),
            "loglik_rel_diff_vs_full": abs(ll_s - ll_f) / abs(ll_f),
            "note": "tiles whose every pair term is an exact FP32 zero are skipped "
                    "(HAWKES_SKIP_UNDERFLOW); not the headline"}

    # the same step evaluating only the tile pairs that can be nonzero in FP32
    # (space-ordered tiles inside time windows; reported separately)
    hk.loglik_grad(p, HAWKES_F32 | HAWKES_SKIP_SPATIAL)  # builds the order (untimed)
    sp_ms = []
    for k in range(args.steps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        hk.resample(2, chain, 900 + k)
        ll_x, g_x = hk.loglik_grad(p, HAWKES_F32 | HAWKES_SKIP_SPATIAL)
        e1.record(stream)
        torch.cuda.synchronize()
        if k:
            sp_ms.append(e0.elapsed_time(e1))
    hk.resample(2, chain, 900 + args.steps)
    ll_y, g_y = hk.loglik_grad(p, HAWKES_F32)
    skip_spatial = {"ms_per_step": sum(sp_ms) / len(sp_ms),
                    "pairs_per_s_equivalent": pairs / (sum(sp_ms) / len(sp_ms) / 1000.0),
                    "speedup": (1000 * T / args.steps) / (sum(sp_ms) / len(sp_ms)),
                    "loglik_rel_diff_vs_full": abs(ll_x - ll_y) / abs(ll_y),
                    "grad_max_rel_diff_vs_full": float(np.max(np.abs(np.asarray(g_x) - np.asarray(g_y)) /
                                                              np.maximum(np.abs(np.asarray(g_y)), 1e-300))),
                    "note": "only tile pairs whose terms can be nonzero in FP32 are evaluated "
                            "(HAWKES_SKIP_SPATIAL: events ordered by location inside time windows of "
                            "131,072 events); same result up to FP32 summation order; not the headline"}

    # the same step with eq. 2's time-only background (a model option, not the headline)
    bgt_ms = []
    for k in range(args.steps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        hk.resample(2, chain, 700 + k)
        hk.loglik_grad(p, HAWKES_F32 | HAWKES_BG_TIME)
        e1.record(stream)
        torch.cuda.synchronize()
        if k:
            bgt_ms.append(e0.elapsed_time(e1))
    bg_time = {"ms_per_step": sum(bgt_ms) / len(bgt_ms),
               "pairs_per_s": pairs / (sum(bgt_ms) / len(bgt_ms) / 1000.0),
               "note": "background mu phi1(dt; tau_t) / tau_x^2 (HAWKES_BG_TIME), same variant; "
                       "a model option, not the headline"}

    # the same step evaluating the log-likelihood only (the paper's own
    # computation, what its univariate Metropolis-Hastings sampler needs)
    ll_ms = []
    hk.profile(True)
    for k in range(args.steps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        hk.resample(2, chain, 1300 + k)
        ll_o, _ = hk.loglik_grad(p, HAWKES_F32 | HAWKES_LOGLIK_ONLY)
        e1.record(stream)
        torch.cuda.synchronize()
        if k:
            ll_ms.append(e0.elapsed_time(e1))
    pll = hk.profile(False)
    hk.resample(2, chain, 1300 + args.steps)
    ll_ref, _ = hk.loglik_grad(p, HAWKES_F32)
    ll_sweep_s = pll["sweep"][1] / max(pll["sweep"][0], 1) / 1000.0
    loglik_only = {"ms_per_step": sum(ll_ms) / len(ll_ms),
                   "pairs_per_s": pairs / (sum(ll_ms) / len(ll_ms) / 1000.0),
                   "sweep_ms": 1000 * ll_sweep_s,
                   "roofline_frac": LL_FP32_OPS_PER_PAIR * pairs / ll_sweep_s / (
                       torch.cuda.get_device_properties(local).multi_processor_count * FP32_LANES_PER_SM *
                       float(peaks()[0].get("sm_max_mhz", 2070.0)) * 1e6),
                   "per_unit": f"{LL_FP32_OPS_PER_PAIR} FP32 lane ops per unordered pair",
                   "loglik_rel_diff_vs_full": abs(ll_o - ll_ref) / abs(ll_ref),
                   "note": "HAWKES_LOGLIK_ONLY: two moment sums per row instead of six, no gradient"}

    # one evaluation split in row-tile shards that keep the symmetric sweep,
    # against the row-window split without it (the split of Sec. 2.3.2), run
    # one after another on this GPU; sweep kernel times only
    shards = {}
    dpar = torch.tensor(p, dtype=torch.float64, device="cuda")
    mom = torch.empty(6 * n, dtype=torch.float64, device="cuda")
    for G in (2, 4):
        per = []
        for gi in range(G):
            hk.shard_moments(dpar.data_ptr(), gi, G, mom.data_ptr())  # builds the shard's list
            hk.profile(True)
            hk.shard_moments(dpar.data_ptr(), gi, G, mom.data_ptr())
            per.append(hk.profile(False)["sweep"][1])
        shards[f"symmetric_{G}_shard_sweep_ms"] = [round(v, 2) for v in per]
    win = []
    for a, b_ in ((0, n // 2), (n // 2, n)):
        hk.profile(True)
        hk.loglik_grad(p, HAWKES_F32, a, b_)
        win.append(hk.profile(False)["sweep"][1])
    shards["row_window_2_shard_sweep_ms"] = [round(v, 2) for v in win]
    shards["whole_sweep_ms"] = round(1000 * sweep_avg_s, 2)
    shards["note"] = ("sweep kernel time of each shard of one N=1M evaluation, run one after another on one "
                      "GPU: symmetric row-tile shards (hawkes_shard_moments, equal pair counts) against "
                      "uniform row windows evaluated without the symmetric shortcut")

    # end to end through the C ABI from pinned host buffers, every step
    pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy()
           for k, v in (("t", ds.t), ("x", ds.x), ("y", ds.y), ("county", ds.county.astype(np.int32)),
                        ("scale", ds.county_scale))}
    h2d = sum(v.nbytes for v in pin.values()) + 48
    d2h = 7 * 8
    hk.set_events(pin["t"], pin["county"], pin["scale"], pin["x"], pin["y"])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        hk.set_events(pin["t"], pin["county"], pin["scale"], pin["x"], pin["y"])
        hk.resample(2, chain, 1000 + k)
        ll_e, g_e = hk.loglik_grad(p, HAWKES_F32)
    torch.cuda.synchronize()
    Te = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([Te], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        Te = float(t.item())
    e2e_value = world * args.e2e_steps * pairs / Te

    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * T / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.workload == "c3" else args.workload, "n_events": n, "pairs_per_step": pairs,
                       "chains": world, "l2": "256 MB buffer written between timed steps",
                       "loglik": ll, "grad": list(map(float, g))},
            "gpu_launches": int(launches),
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in prof.items() if v[0]},
            "roofline": {"bound": "alu", "achieved": achieved_ops / 1e12, "peak": peak_ops / 1e12,
                         "unit": "Top/s", "frac": achieved_ops / peak_ops,
                         "traffic": profiled_traffic(),
                         "kernel": f"k_sweep variant {variant} (FP32 pair sweep)",
                         "tuned_ms": [round(float(x), 3) for x in tune_ms],
                         "per_unit": f"{ALG_FP32_OPS_PER_PAIR} FP32 lane ops per unordered pair",
                         "frac_at_24_ops_per_pair": ESTIMATED_FP32_OPS_PER_PAIR * pairs / sweep_avg_s / peak_ops,
                         "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_mhz:.0f} MHz "
                                        f"(sm_max_mhz, {pk_src})",
                         "launch_ms": 1000 * sweep_avg_s},
            "clocks": clk.summary(),
            "skip_underflow": skip,
            "skip_spatial": skip_spatial,
            "bg_time": bg_time,
            "loglik_only": loglik_only,
            "shards": shards,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": args.e2e_steps},
        }
        if args.workload == "c3":
            acc = accuracy_c3(hk, ds, p)
            out["accuracy"] = acc
            if acc.get("rel_err"):
                out["accuracy_loglik_rel_err"] = acc["rel_err"]["loglik"]
                out["accuracy_grad_max_rel_err"] = max(v for k, v in acc["rel_err"].items() if k != "loglik")
        out["loglik_only_ms_per_step"] = loglik_only["ms_per_step"]
        out["skip_spatial_ms_per_step"] = skip_spatial["ms_per_step"]
        if world == 1 and not args.no_batch and args.workload == "c3":
            bt = bench_batch(ds, steps=args.batch_repeats, warmup=1)
            out["batch30"] = bt
            out["batch30_speedup"] = bt["speedup_vs_sequential"]
            out["batch30_speedup_min_max"] = [bt["speedup_min"], bt["speedup_max"]]
            out["batch30_chains_per_cta"] = bt["tuned"]["chains_per_cta"]
        if world == 1 and args.hmc_n > 0 and args.workload == "c3":
            out["hmc"] = {"cut_posterior": bench_hmc(args.hmc_n, cut=True, ref_rounds=args.hmc_cut_reference),
                          "fixed_locations": bench_hmc(args.hmc_n, cut=False)}
            out["hmc_cut_surrogate_ess_per_s_ratio"] = out["hmc"]["cut_posterior"]["speedup_ess_per_s"]
            out["hmc_fixed_surrogate_ess_per_s_ratio"] = out["hmc"]["fixed_locations"]["speedup_ess_per_s"]
            out["hmc_cut_feature_surrogate_ess_per_s_ratio"] = \
                out["hmc"]["cut_posterior"]["surrogate_feature"]["ess_per_s_vs_exact"]
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(ds)
        print(json.dumps(out))
    hk.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
