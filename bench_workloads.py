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
  visual        line charts on an 800 x 250 canvas: rasteriser throughput on the chart of
                all points of a 1e7 float32 walk + sines + spikes; and for a 2e5-point
                template of the same kind (the reference-image size of the paper's figure)
                the charts of MinMax, MinMaxLTTB (r_ps 2, 4, 6, 8), LTTB and M4 at n_out
                200..2000 with their PEM_20 and MSE against the chart of all points.
"""
import ctypes
import json
import time

import numpy as np
import torch

import synth


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
    nmed, nmean = _time_calls(lambda: f(ctypes.c_void_p(y.data_ptr()), 0, None, 0, ctypes.c_int64(n),
                                        ctypes.c_int64(n_out), ctypes.c_int32(r_ps), 0,
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_int64(n_out), None,
                                        ctypes.c_void_p(st)), args.steps)
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


def run_1e8(args, mm):
    n = 100_000_000
    y = torch.from_numpy(synth.walk_sines_spikes(n, seed=0)).cuda()
    res = {}
    for r_ps in (2, 4, 8, 16):
        med, _ = _time_calls(lambda: mm.minmaxlttb(y, 2000, r_ps, sync=False), max(10, args.steps // 10))
        res[f"minmaxlttb_r{r_ps}_ms"] = med
    lt, _ = _time_calls(lambda: mm.lttb(y, 2000, sync=False), 5, warmup=2)
    res["plain_lttb_ms"] = lt
    speed = lt / res["minmaxlttb_r4_ms"]
    _line("MinMaxLTTB (r_ps=4) speedup over plain GPU LTTB at n_in=1e8", speed, "x", True,
          {"workload": "single series n_in=1e8 float32 walk + sines + spikes, n_out=2000"},
          {"dtype": "f32", **res, "minmaxlttb_r4_gpts_per_s": n / (res["minmaxlttb_r4_ms"] * 1e-3) / 1e9}, args)


def run_batched(args, mm):
    lens, nouts = synth.batch_shapes(4096, seed=0)
    t = time.time()
    ys = [torch.from_numpy(synth.random_walk(int(k), seed=1000 + i, dtype=np.float32)).cuda()
          for i, k in enumerate(lens)]
    gen = time.time() - t
    total = int(lens.sum())
    b = mm.Batch([{"y": y, "n_out": int(k), "r_ps": 4} for y, k in zip(ys, nouts)])
    steps = max(5, args.steps // 50)
    gmed, gmean = _time_calls(lambda: b.run(graph=True), steps, warmup=3)
    # 4096 single-series calls, everything preallocated, back to back on one stream
    lib = mm.lib
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = [torch.empty(max(1, min(int(k), int(n))), dtype=torch.int64, device="cuda") for k, n in zip(nouts, lens)]
    wss = [torch.empty(mm.workspace_bytes(mm.OP_MINMAXLTTB, mm.F32, mm.X_IMPLICIT, int(n), int(k), 4),
                       dtype=torch.uint8, device="cuda") for k, n in zip(nouts, lens)]
    calls = [(ctypes.c_void_p(y.data_ptr()), ctypes.c_int64(int(n)), ctypes.c_int64(int(k)),
              ctypes.c_void_p(o.data_ptr()), ctypes.c_int64(o.numel()), ctypes.c_void_p(w.data_ptr()),
              ctypes.c_size_t(w.numel())) for y, n, k, o, w in zip(ys, lens, nouts, outs, wss)]
    f = lib.mmlttb_minmaxlttb

    def singles():
        for yp, n, k, op, cap, wp, wb in calls:
            f(yp, 0, None, 0, n, k, 4, 0, op, cap, None, wp, wb, st)
    smed, _ = _time_calls(singles, 3, warmup=1)
    res = b.results()
    same = all(torch.equal(res[i][: outs[i].numel()], outs[i][: res[i].numel()]) for i in range(0, 4096, 97))
    _line("batched MinMaxLTTB throughput, 4096 series (Gpts/s)", total / (gmed * 1e-3) / 1e9, "Gpts/s", True,
          {"workload": "4096 float32 walks, lengths round(10^U(3,7)), n_out U{200..4000}, r_ps=4",
           "total_points": total},
          {"dtype": "f32", "graph_ms": gmed, "singles_ms": smed, "speedup_vs_singles": smed / gmed,
           "singles_gpts_per_s": total / (smed * 1e-3) / 1e9, "sample_equal": same,
           "input_gen_s": round(gen, 1)}, args)


def run_serving(args, mm):
    S, n = 64, 100_000_000
    t = time.time()
    ys = [torch.from_numpy(synth.random_walk(n, seed=5000 + i, dtype=np.float32)).cuda() for i in range(S)]
    gen = time.time() - t
    rng = np.random.default_rng(0)
    rates = [1000, 5000, 10000, 20000, 50000, 100000, 150000]
    duration = 1.0
    results = {}

    def trace(rate, rng=rng):
        k = int(rate * duration)
        offs = np.cumsum(rng.exponential(1.0 / rate, k))
        width = np.rint(10 ** rng.uniform(4, 8, k)).astype(np.int64)
        start = (rng.random(k) * (n - width + 1)).astype(np.int64)
        sid = rng.integers(0, S, k)
        nout = rng.integers(500, 4001, k)
        return [mm.Request(int(a), int(b), int(b + w), int(c), 4, 0) for a, b, w, c in
                zip(sid, start, width, nout)], offs.tolist()

    for mode, cfg in (("batched", dict(streams=3, max_batch=256, workspace_bytes_per_stream=1 << 30)),
                      ("per_request", dict(streams=1, max_batch=1, workspace_bytes_per_stream=64 << 20))):
        srv = mm.Server(max_pending=1 << 22, **cfg)
        for y in ys:
            srv.add_series(y)
        # warm-up (untimed, its own random stream): the first launches of every kernel
        wreqs, woffs = trace(2000, np.random.default_rng(1))
        wids, _ = srv.replay(wreqs[:400], woffs[:400])
        srv.drain()
        for i in wids:
            if i:
                srv.wait(i)
        for rate in rates:
            reqs, offs = trace(rate)
            if mode == "per_request" and rate > 50000:
                continue  # saturated near 1e4 req/s: these traces would only queue
            srv.reset_stats()
            t0 = time.perf_counter()
            ids, st = srv.replay(reqs, offs)
            srv.drain()
            el = time.perf_counter() - t0
            s = srv.stats()
            results[f"{mode}@{rate}"] = {"offered_rps": rate, "achieved_rps": s["completed"] / el,
                                          "p50_ms": s["latency_p50_s"] * 1e3, "p99_ms": s["latency_p99_s"] * 1e3,
                                          "mean_batch": s["mean_batch"], "completed": s["completed"]}
            for i in ids:
                if i:
                    srv.wait(i)
        srv.close()
    best = max((v["achieved_rps"] for k, v in results.items() if k.startswith("batched") and v["p99_ms"] < 100.0),
               default=0.0)
    _line("served zoom requests per second with p99 latency under 100 ms", best, "req/s", True,
          {"workload": "64 x 1e8 float32 resident walks; Poisson windows, width log-U[1e4,1e8], "
                       "n_out U{500..4000}, r_ps=4"},
          {"dtype": "f32", "rates": results, "input_gen_s": round(gen, 1)}, args)


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
                            "kind": "oracle", "sample": f"chart of the first {S} points, single-threaded C oracle"}},
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
     "visual": run_visual}[args.workload](args, mm)
