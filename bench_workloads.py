"""The other measured MinMaxLTTB workloads (bench.py --workload ...), one JSON line each.

  1e6           single series, 1e6 float32 walk points, n_out=1000, r_ps=4: latency of one
                call (device events), plus the same call replayed as a CUDA graph and the
                allocation-free entry point.
  1e8-vs-lttb   1e8 float32 walk + sines + spikes, n_out=2000: MinMaxLTTB for r_ps in
                {2,4,8,16} against plain LTTB on all points, on the same GPU.
  batched-4096  4096 float32 walks, lengths round(10^U(3,7)), n_out in U{200..4000}, r_ps=4:
                one batched launch sequence replayed as a CUDA graph vs 4096 single calls.
  serving       64 resident series of 1e8 float32 points; Poisson zoom-window requests
                (width log-uniform in [1e4, 1e8], n_out in U{500..4000}, r_ps=4) at several
                rates; continuous-batching server vs one request per launch; p50/p99.
  bins          MinMax stream rate by index-bin size (16 to 25 000 points) on 1e8 float32
                walk points, register stream against the staged (cp.async.bulk) stream.
  visual        line charts on an 800 x 250 canvas: rasteriser throughput on the chart of
                all points of a 1e7 float32 walk + sines + spikes; and for a 2e5-point
                template of the same kind (the reference-image size of the paper's figure)
                the charts of MinMax, MinMaxLTTB (r_ps 2, 4, 6, 8), LTTB and M4 at n_out
                200..2000 with their PEM_20 and MSE against the chart of all points.
"""
import contextlib
import ctypes
import json
import os
import platform
import subprocess
import time

import numpy as np
import torch

import synth


def host_cpu():
    """The host's CPU model and core count, for the oracle timings."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"cpu_model": model or platform.machine(), "nproc": os.cpu_count()}


@contextlib.contextmanager
def one_core():
    """Pin the calling thread to one core (the last it may run on) for an oracle timing;
    yields the core, or None where affinity cannot be set."""
    try:
        old = os.sched_getaffinity(0)
        core = max(old)
        os.sched_setaffinity(0, {core})
    except (AttributeError, OSError, ValueError):
        old, core = None, None
    try:
        yield core
    finally:
        if old is not None:
            os.sched_setaffinity(0, old)


def _events(n):
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    for e in ev:
        e.record()
    return ev


def _time_calls(fn, steps, warmup=5):
    """Per-call device time (median, ms) and back-to-back mean (ms) of fn()."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = _events(steps + 1)
    torch.cuda.synchronize()
    for i in range(steps):
        ev[i].record()
        fn()
    ev[steps].record()
    torch.cuda.synchronize()
    per = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(steps))
    return per[len(per) // 2], ev[0].elapsed_time(ev[steps]) / steps


def _line(metric, value, unit, hib, config, extra, args):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
         "warmup": args.warmup, "higher_is_better": hib, "scaling": "weak", "vs_baseline": None,
         "data": "synthetic", "config": config}
    d.update(extra)
    print(json.dumps(d), flush=True)


def run_1e6(args, mm):
    n, n_out, r_ps = 1_000_000, 1000, 4
    y = torch.from_numpy(synth.random_walk(n, seed=0, dtype=np.float32)).cuda()
    out = torch.empty(n_out, dtype=torch.int64, device="cuda")
    ws = torch.empty(mm.workspace_bytes(mm.OP_MINMAXLTTB, mm.F32, mm.X_IMPLICIT, n, n_out, r_ps),
                     dtype=torch.uint8, device="cuda")
    med, mean = _time_calls(lambda: mm.minmaxlttb(y, n_out, r_ps, out=out, workspace=ws, sync=False),
                            args.steps)
    b = mm.Batch([{"y": y, "n_out": n_out, "r_ps": r_ps}])
    gmed, gmean = _time_calls(lambda: b.run(graph=True), args.steps)
    f = mm.lib.mmlttb_minmaxlttb_noalloc
    f.restype = ctypes.c_int
    st = torch.cuda.current_stream().cuda_stream

    def noalloc():
        return f(ctypes.c_void_p(y.data_ptr()), 0, None, 0, ctypes.c_int64(n), ctypes.c_int64(n_out),
                 ctypes.c_int32(r_ps), 0, ctypes.c_void_p(out.data_ptr()), ctypes.c_int64(n_out), None,
                 ctypes.c_void_p(st))
    out.fill_(-1)
    rc = noalloc()  # untimed: the call must succeed and equal the workspace entry point
    if rc != mm.OK:
        raise RuntimeError(f"mmlttb_minmaxlttb_noalloc: {mm.strerror(rc)}")
    if not torch.equal(out, mm.minmaxlttb(y, n_out, r_ps)):
        raise RuntimeError("mmlttb_minmaxlttb_noalloc disagrees with mmlttb_minmaxlttb")
    nmed, nmean = _time_calls(noalloc, args.steps)
    paths = {}
    for name, pid in (("split", mm.PATH_SPLIT), ("fused_tail", mm.PATH_FUSED_TAIL), ("fused", mm.PATH_FUSED)):
        mm.set_single_path(pid)
        pm, pb = _time_calls(lambda: mm.minmaxlttb(y, n_out, r_ps, out=out, workspace=ws, sync=False),
                             args.steps)
        paths[name] = {"us": pm * 1e3, "us_back_to_back": pb * 1e3}
    mm.set_single_path(mm.PATH_AUTO)
    _line("MinMaxLTTB latency of one call at n_in=1e6 (device time)", med * 1e3, "us", False,
          {"workload": "single series n_in=1e6 float32 walk, implicit x, n_out=1000, r_ps=4, index bins"},
          {"dtype": "f32", "us_back_to_back": mean * 1e3, "graph_us": gmed * 1e3,
           "graph_us_back_to_back": gmean * 1e3, "noalloc_us": nmed * 1e3,
           "launch_path": "auto", "by_path": paths,
           "gpts_per_s_back_to_back": n / (mean * 1e-3) / 1e9}, args)


def _per_step_ms(fn, steps, warmup):
    """CUDA-event device time of each of `steps` calls of fn() after `warmup` untimed
    calls (events on the current stream, a synchronize on both sides)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = _events(steps + 1)
    torch.cuda.synchronize()
    for i in range(steps):
        ev[i].record()
        fn()
    ev[steps].record()
    torch.cuda.synchronize()
    return [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]


def _med(v):
    v = sorted(v)
    return v[len(v) // 2]


def _clocks(index):
    from bench import ClockSampler
    c = ClockSampler(index)
    c.start()
    time.sleep(0.3)
    return c


def _peak_gbs():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def record_vs_plain_lttb(mm, steps, warmup, clock_index="0", oracle=True):
    """1e8 float32 walk + sines + spikes, n_out = 2000: MinMaxLTTB at r_ps 2, 4, 8, 16
    against plain LTTB on all points, on the same GPU (device events per call)."""
    n, n_out = 100_000_000, 2000
    t = time.time()
    y_h = synth.walk_sines_spikes(n, seed=0)
    gen = time.time() - t
    y = torch.from_numpy(y_h).cuda()
    out = torch.empty(n_out, dtype=torch.int64, device="cuda")
    wsb = max([mm.workspace_bytes(mm.OP_MINMAXLTTB, mm.F32, mm.X_IMPLICIT, n, n_out, r) for r in (2, 4, 8, 16)]
              + [mm.workspace_bytes(mm.OP_LTTB, mm.F32, mm.X_IMPLICIT, n, n_out)])
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    clk = _clocks(clock_index)
    t0 = time.time()
    per = {}
    for r_ps in (2, 4, 8, 16):
        per[r_ps] = _per_step_ms(lambda: mm.minmaxlttb(y, n_out, r_ps, out=out, workspace=ws, sync=False),
                                 steps, warmup)
    plain = _per_step_ms(lambda: mm.lttb(y, n_out, out=out, workspace=ws, sync=False), steps, warmup)
    t1 = time.time()
    clk.stop()
    r4 = _med(per[4])
    rec = {"workload": "single series n_in=1e8 float32 walk + sines (periods 1e3/1e5/1e7) + spikes, "
                       "implicit x, n_out=2000, index bins",
           "n_in": n, "n_out": n_out, "steps": steps, "warmup": warmup, "dtype": "f32",
           "minmaxlttb_ms": {str(r): _med(v) for r, v in per.items()},
           "plain_lttb_ms": _med(plain), "plain_lttb_ms_mean": sum(plain) / len(plain),
           "speedup_r4_vs_plain_lttb": _med(plain) / r4,
           "minmaxlttb_r4_gpts_per_s": n / (r4 * 1e-3) / 1e9,
           "plain_lttb_gpts_per_s": n / (_med(plain) * 1e-3) / 1e9,
           "clocks": clk.summary(t0, t1), "input_gen_s": round(gen, 1)}
    if oracle:
        from oracle import oracle as load_oracle
        o = load_oracle()
        g4 = mm.minmaxlttb(y, n_out, 4).cpu().numpy()
        gp = mm.lttb(y, n_out).cpu().numpy()
        with one_core() as core:
            t = time.perf_counter()
            e4 = o.minmaxlttb(y_h, n_out, 4)
            c4 = time.perf_counter() - t
            t = time.perf_counter()
            ep = o.lttb(y_h, n_out)
            cp = time.perf_counter() - t
        ok = np.array_equal(g4, e4) and np.array_equal(gp, ep)
        rec["parity_vs_oracle"] = "bit-exact" if ok else "MISMATCH"
        rec["cpu_baseline"] = {"value": n / c4 / 1e9, "unit": "Gpts/s", "cores": 1, "kind": "oracle",
                               "sample": "the full 1e8-point series once, MinMaxLTTB r_ps=4, single-threaded C oracle",
                               "plain_lttb_s": cp, "pinned_core": core, **host_cpu()}
    del y, ws
    torch.cuda.empty_cache()
    return rec


def run_1e8(args, mm):
    rec = record_vs_plain_lttb(mm, max(5, args.steps // 10), max(3, args.warmup))
    _line("MinMaxLTTB (r_ps=4) speedup over plain GPU LTTB at n_in=1e8", rec["speedup_r4_vs_plain_lttb"], "x",
          True, {"workload": rec["workload"]}, rec, args)


BATCH_SEED = 1000


def record_batched(mm, steps, warmup, clock_index="0", oracle=True, singles_reps=3, n_series=4096):
    """4096 float32 walks, lengths round(10^U(3,7)), n_out U{200..4000}, r_ps = 4: one
    batched launch sequence replayed as a CUDA graph, against 4096 single calls.  With
    n_series < 4096, the first n_series of those series (a smaller case of the same
    mix, for profiling)."""
    lens, nouts = synth.batch_shapes(4096, seed=0)
    lens, nouts = lens[:n_series], nouts[:n_series]
    t = time.time()
    ys_h = synth.random_walks(lens, BATCH_SEED)
    gen = time.time() - t
    ys = [torch.from_numpy(v).cuda() for v in ys_h]
    total = int(lens.sum())
    sample = sorted(set(np.random.default_rng(1).choice(n_series, min(48, n_series), replace=False).tolist())
                    | set(np.argsort(lens)[-4:].tolist()))
    ys_h = {i: ys_h[i] for i in sample}  # the host copies the oracle sample needs
    b = mm.Batch([{"y": y, "n_out": int(k), "r_ps": 4} for y, k in zip(ys, nouts)])
    tuning = b.tuning()  # the tuple the batch was planned with
    # kernel breakdown of one uncaptured run (stage events at fixed points)
    names = ["upload", "edges", "stream", "compaction", "tables", "chain", "block"]
    stage = {k: [] for k in names[1:]}
    for _ in range(max(3, warmup)):
        b.run(graph=False)
    for _ in range(5):
        ev = _events(len(names))
        torch.cuda.synchronize()
        mm.set_stage_events(ev)
        b.run(graph=False)
        torch.cuda.synchronize()
        for k in range(1, len(names)):
            stage[names[k]].append(ev[k - 1].elapsed_time(ev[k]))
    stage_ms = {k: _med(v) for k, v in stage.items()}
    # the stream kernel reads every interior point of the series that take the
    # MinMax branch (r_ps * n_out < n); the other series are read by the LTTB kernels
    binned = [int(n) for n, k in zip(lens, nouts) if 4 * int(k) < int(n)]
    stream_bytes = 4 * sum(n - 2 for n in binned)
    peak, peak_src = _peak_gbs()
    clk = _clocks(clock_index)
    t0 = time.time()
    per = _per_step_ms(lambda: b.run(graph=True), steps, warmup)
    t1 = time.time()
    # 4096 single-series calls, everything preallocated, back to back on one stream
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = [torch.empty(max(1, min(int(k), int(n))), dtype=torch.int64, device="cuda") for k, n in zip(nouts, lens)]
    wss = [torch.empty(mm.workspace_bytes(mm.OP_MINMAXLTTB, mm.F32, mm.X_IMPLICIT, int(n), int(k), 4),
                       dtype=torch.uint8, device="cuda") for k, n in zip(nouts, lens)]
    calls = [(ctypes.c_void_p(y.data_ptr()), ctypes.c_int64(int(n)), ctypes.c_int64(int(k)),
              ctypes.c_void_p(o.data_ptr()), ctypes.c_int64(o.numel()), ctypes.c_void_p(w.data_ptr()),
              ctypes.c_size_t(w.numel())) for y, n, k, o, w in zip(ys, lens, nouts, outs, wss)]
    f = mm.lib.mmlttb_minmaxlttb

    def singles():
        for yp, n, k, op, cap, wp, wb in calls:
            rc = f(yp, 0, None, 0, n, k, 4, 0, op, cap, None, wp, wb, st)
            if rc:
                raise RuntimeError(mm.strerror(rc))
    t2 = time.time()
    sper = _per_step_ms(singles, singles_reps, 1)
    t3 = time.time()
    clk.stop()
    res = b.results()
    same = all(torch.equal(res[i], outs[i][: res[i].numel()]) and res[i].numel() == outs[i].numel()
               for i in range(n_series))
    g = _med(per)
    unroll, min_blocks = mm.stream_variants()[tuning["variant"]]
    variant = {"tuning": tuning, "loads_in_flight_per_lane": unroll, "ctas_per_sm": min_blocks,
               "threads_per_cta": mm.stream_variant_threads(tuning["variant"])}
    what = "4096 float32 walks" if n_series == 4096 else f"the first {n_series} of the 4096 float32 walks"
    rec = {"workload": what + ", lengths round(10^U(3,7)), n_out U{200..4000}, r_ps=4, implicit x",
           "total_points": total, "steps": steps, "warmup": warmup, "dtype": "f32",
           "graph_ms": g, "graph_ms_mean": sum(per) / len(per), "gpts_per_s": total / (g * 1e-3) / 1e9,
           "singles_ms": _med(sper), "singles_gpts_per_s": total / (_med(sper) * 1e-3) / 1e9,
           "speedup_vs_singles": _med(sper) / g, "batch_equals_singles": same,
           "stage_ms_uncaptured": stage_ms,
           "roofline": {"bound": "hbm", "kernel": "k_stream inside the batch (MinMax preselection)",
                        "achieved": stream_bytes / (stage_ms["stream"] * 1e-3) / 1e9, "peak": peak,
                        "peak_source": peak_src, "unit": "GB/s",
                        "frac": stream_bytes / (stage_ms["stream"] * 1e-3) / 1e9 / peak,
                        "algorithmic_bytes_per_launch": stream_bytes, "traffic": None},
           "whole_batch_hbm_frac": 4 * total / (g * 1e-3) / 1e9 / peak,
           "stream_variant": variant,
           "l2": "no flush: 18.4 GB of series per step exceed L2 (129 MB)",
           "clocks": clk.summary(t0, t3), "input_gen_s": round(gen, 1)}
    if oracle:
        from oracle import oracle as load_oracle
        o = load_oracle()
        pts, el, ok = 0, 0.0, True
        exp = {}
        with one_core() as core:
            for i in sample:
                t = time.perf_counter()
                exp[i] = o.minmaxlttb(ys_h[i], int(nouts[i]), 4)
                el += time.perf_counter() - t
                pts += int(lens[i])
        for i in sample:
            ok &= bool(np.array_equal(res[i].cpu().numpy(), exp[i]))
        rec["parity_vs_oracle"] = ("bit-exact" if ok else "MISMATCH") + f" on {len(sample)} sampled series"
        rec["cpu_baseline"] = {"value": pts / el / 1e9, "unit": "Gpts/s", "cores": 1, "kind": "oracle",
                               "sample": f"{len(sample)} seeded series of the batch ({pts} points), "
                                         "single-threaded C oracle", "pinned_core": core, **host_cpu()}
    b.close()
    del ys, outs, wss, res
    torch.cuda.empty_cache()
    return rec


def run_batched(args, mm):
    rec = record_batched(mm, max(5, args.steps // 10), max(3, args.warmup), n_series=args.series)
    _line(f"batched MinMaxLTTB throughput, {args.series} series (Gpts/s)", rec["gpts_per_s"], "Gpts/s", True,
          {"workload": rec["workload"], "total_points": rec["total_points"]}, rec, args)


def run_bins(args, mm):
    """MinMax stream rate by index-bin size on 1e8 float32 walk points (preselection,
    r_ps = 2, n_out = points per bin / (n - 2)): the register stream and the staged
    (cp.async.bulk) stream, CUDA events around the stream kernel, the same indices."""
    n = 100_000_000
    y = torch.from_numpy(synth.random_walk(n, seed=3, dtype=np.float32)).cuda()
    sizes = [args.bin_points] if args.bin_points else [16, 64, 125, 256, 1024, 4096, 25000]
    rows = []
    clk = _clocks("0")
    t0 = time.time()
    for S in sizes:
        n_out = max(3, int((n - 2) / S))
        row = {"points_per_bin": S}
        outs = {}
        for staged in (False, True):
            mm.set_stream_staging(staged)
            tiles = mm.stream_tiles(mm.OP_PRESELECT, mm.F32, mm.X_IMPLICIT, n, n_out, 2)
            if staged and tiles == 0:
                row["staged_gbs"] = None  # bins too large for the staged stream
                continue
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            b.record()
            ts = []
            for r in range(max(3, args.warmup) + max(3, args.steps)):
                mm.set_timing_events(a, b)
                outs[staged] = mm.minmax_preselect(y, n_out, 2)
                torch.cuda.synchronize()
                if r >= max(3, args.warmup):
                    ts.append(a.elapsed_time(b))
            row["staged_gbs" if staged else "register_gbs"] = 4 * (n - 2) / (_med(ts) * 1e-3) / 1e9
        mm.set_stream_staging(False)
        row["same_indices"] = len(outs) < 2 or bool(torch.equal(outs[False], outs[True]))
        rows.append(row)
    t1 = time.time()
    clk.stop()
    peak, peak_src = _peak_gbs()
    best = max(max(r["register_gbs"], r["staged_gbs"] or 0) for r in rows)
    _line("MinMax stream rate by bin size, 1e8 float32 points (GB/s)", best, "GB/s", True,
          {"workload": "1e8 float32 walk, MinMax preselection r_ps=2, index bins of the given points"},
          {"rows": rows, "peak": peak, "peak_source": peak_src, "dtype": "f32",
           "l2": "no flush: 400 MB of y per step exceed L2 (129 MB)", "clocks": clk.summary(t0, t1)}, args)


SERVE_SEED = 5000


def record_serving(mm, clock_index="0", rates=(5000, 20000, 50000), repeats=3, duration=1.0,
                   per_request_rates=(5000, 20000), n_series=64, n=100_000_000):
    """64 resident float32 walks of 1e8 points; Poisson zoom-window requests (width
    log-uniform in [1e4, 1e8], n_out U{500..4000}, r_ps = 4); a continuous-batching
    server (3 streams, up to 256 requests per batch) against one request per launch.
    Each rate is replayed `repeats` times with fresh arrivals."""
    t = time.time()
    ys = []
    for i in range(n_series):  # one host series at a time: the pool lives on the device
        ys.append(torch.from_numpy(synth.random_walk(n, seed=SERVE_SEED + i, dtype=np.float32)).cuda())
    gen = time.time() - t
    rng = np.random.default_rng(0)

    def trace(rate, rng):
        k = int(rate * duration)
        offs = np.cumsum(rng.exponential(1.0 / rate, k))
        width = np.rint(10 ** rng.uniform(4, 8, k)).astype(np.int64)
        start = (rng.random(k) * (n - width + 1)).astype(np.int64)
        sid = rng.integers(0, n_series, k)
        nout = rng.integers(500, 4001, k)
        return [mm.Request(int(a), int(b), int(b + w), int(c), 4, 0) for a, b, w, c in
                zip(sid, start, width, nout)], offs.tolist()

    out = {}
    checked, agree = 0, True
    clk = _clocks(clock_index)
    t0 = time.time()
    for mode, cfg, mode_rates in (
            ("batched", dict(streams=3, max_batch=256, workspace_bytes_per_stream=1 << 30), rates),
            ("per_request", dict(streams=1, max_batch=1, workspace_bytes_per_stream=64 << 20), per_request_rates)):
        srv = mm.Server(max_pending=1 << 22, **cfg)
        for y in ys:
            srv.add_series(y)
        wreqs, woffs = trace(2000, np.random.default_rng(1))  # untimed warm-up
        wids, _ = srv.replay(wreqs[:400], woffs[:400])
        srv.drain()
        for i in wids:
            if i:
                srv.wait(i)
        for rate in mode_rates:
            runs = []
            for rep in range(repeats):
                reqs, offs = trace(rate, rng)
                srv.reset_stats()
                t_a = time.perf_counter()
                ids, st = srv.replay(reqs, offs)
                srv.drain()
                el = time.perf_counter() - t_a
                s = srv.stats()
                runs.append({"achieved_rps": s["completed"] / el, "p50_ms": s["latency_p50_s"] * 1e3,
                             "p99_ms": s["latency_p99_s"] * 1e3, "mean_batch": s["mean_batch"],
                             "overlapped_batches": s["overlapped_batches"],
                             "max_batches_in_flight": s["max_batches_in_flight"],
                             "completed": s["completed"], "rejected": s["rejected"]})
                for k, (q, i) in enumerate(zip(reqs, ids)):
                    if not i:
                        continue
                    got = srv.wait(i)[0]
                    if mode == "batched" and rep == 0 and k % max(1, len(reqs) // 8) == 0:
                        y = ys[q.series][q.start:q.end]
                        exp = mm.minmaxlttb(y, q.n_out, q.r_ps).cpu().numpy() + q.start
                        agree &= bool(np.array_equal(got, exp))
                        checked += 1
            out[f"{mode}@{rate}"] = {
                "offered_rps": rate, "repeats": repeats,
                **{f"{key}_median": _med([r[key] for r in runs]) for key in ("achieved_rps", "p50_ms", "p99_ms")},
                **{f"{key}_min": min(r[key] for r in runs) for key in ("achieved_rps", "p50_ms", "p99_ms")},
                **{f"{key}_max": max(r[key] for r in runs) for key in ("achieved_rps", "p50_ms", "p99_ms")},
                "mean_batch_median": _med([r["mean_batch"] for r in runs]),
                "overlapped_batches_median": _med([r["overlapped_batches"] for r in runs]),
                "runs": runs}
        srv.close()
    t1 = time.time()
    clk.stop()
    del ys
    torch.cuda.empty_cache()
    return {"workload": f"{n_series} x {n:.0e} float32 resident walks; Poisson zoom windows, width "
                        "log-U[1e4,1e8], start uniform, n_out U{500..4000}, r_ps=4; 1 s of arrivals per run",
            "modes": {"batched": "continuous batching: 3 streams, up to 256 requests per batch, admission by "
                                 "workspace bytes (1 GiB per stream)",
                      "per_request": "one request per launch sequence on one stream"},
            "rates": out, "results_checked_against_single_calls": checked,
            "results_equal_single_calls": agree, "clocks": clk.summary(t0, t1), "input_gen_s": round(gen, 1)}


def run_serving(args, mm):
    rec = record_serving(mm)
    best = max((v["achieved_rps_median"] for k, v in rec["rates"].items()
                if k.startswith("batched") and v["p99_ms_max"] < 100.0), default=0.0)
    _line("served zoom requests per second with p99 latency under 100 ms", best, "req/s", True,
          {"workload": rec["workload"]}, rec, args)


def run_visual(args, mm):
    n, W, H = 10_000_000, 800, 250
    y_host = synth.walk_sines_spikes(n, seed=0)
    y = torch.from_numpy(y_host).cuda()
    ext = (0.0, float(n - 1), float(y_host.min()), float(y_host.max()))
    mask = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    mm.raster(y, ext, W, H, mask=mask)
    # OR-ing the same chart into the finished canvas repeats exactly the same work
    steps = max(5, args.steps // 10)
    before = mm.launch_count()
    rmed, rmean = _time_calls(lambda: mm.raster(y, ext, W, H, mask=mask), steps)
    launches = (mm.launch_count() - before) // (steps + 5)
    inked = int((mm.intensity(mask) > 0).sum().item())
    # PEM_20 / MSE table on a 2e5-point template
    nt = 200_000
    t_host = synth.walk_sines_spikes(nt, seed=1, periods=(1e2, 1e4, 1e6))
    yt = torch.from_numpy(t_host).cuda()
    ext_t = (0.0, float(nt - 1), float(t_host.min()), float(t_host.max()))
    ref_img = mm.intensity(mm.raster(yt, ext_t, W, H))
    table = {}
    methods = [("minmax", lambda k: mm.minmax_preselect(yt, k, 1))]
    methods += [(f"minmaxlttb_r{r}", (lambda r: lambda k: mm.minmaxlttb(yt, k, r))(r)) for r in (2, 4, 6, 8)]
    methods += [("lttb", lambda k: mm.lttb(yt, k)), ("m4", lambda k: mm.m4(yt, k))]
    img_mask = torch.zeros_like(mask)
    for name, sel_fn in methods:
        row = {}
        for n_out in (200, 500, 1000, 2000):
            sel = sel_fn(n_out)
            img_mask.zero_()
            mm.raster(yt, ext_t, W, H, idx=sel, mask=img_mask)
            m = mm.visual_metrics(ref_img, mm.intensity(img_mask), 20)
            row[str(n_out)] = {"pem20": round(m["pem"], 5), "mse": round(m["mse"], 2)}
        table[name] = row
    chart_ms = {}
    sel = mm.minmaxlttb(yt, 1000, 4)

    def chart():
        img_mask.zero_()
        mm.raster(yt, ext_t, W, H, idx=sel, mask=img_mask)
        mm.visual_counts(ref_img, mm.intensity(img_mask), 20, sync=False)
    cmed, _ = _time_calls(chart, args.steps)
    chart_ms["minmaxlttb_r4_n_out1000_chart_and_metrics_us"] = cmed * 1e3
    # CPU oracle on a bounded sample: the chart of the first 1e6 points
    from oracle import oracle
    o = oracle()
    S = 1_000_000
    with one_core() as core:
        t = time.perf_counter()
        o.raster(y_host[:S], ext, W, H)
        cpu_s = time.perf_counter() - t
    _line("reference line-chart rasterisation throughput (1e7 points, 800x250, 4x4 samples)",
          (n - 1) / (rmed * 1e-3) / 1e9, "Gsegments/s", True,
          {"workload": "line charts 800x250: 1e7-point float32 walk + sines + spikes (throughput); "
                       "2e5-point template and its downsampled charts, n_out 200..2000 (PEM_20, MSE)"},
          {"dtype": "f32", "reference_chart_ms": rmed, "reference_chart_ms_back_to_back": rmean,
           "inked_pixels": inked, "gpu_launches": launches, **chart_ms, "pem20_mse_template_2e5": table,
           "cpu_baseline": {"value": (S - 1) / cpu_s / 1e9, "unit": "Gsegments/s", "cores": 1,
                            "kind": "oracle", "sample": f"chart of the first {S} points, single-threaded C oracle",
                            "pinned_core": core, **host_cpu()}},
          args)


def run(args):
    import importlib.util
    import os
    root = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("_mmlttb_build", os.path.join(root, "paper_2305_00332_gb300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build_library()
    import paper_2305_00332_gb300 as mm
    torch.cuda.set_device(0)
    {"1e6": run_1e6, "1e8-vs-lttb": run_1e8, "batched-4096": run_batched, "serving": run_serving,
     "visual": run_visual, "bins": run_bins}[args.workload](args, mm)
