"""Benchmark: local energies per second of the symmetry-masked autoregressive
VMC hot path on one GB300 (under torchrun: N data-parallel ranks, one per
GPU, each with its own sample set, exchanging energy statistics and
gradients).

One step = one pass of the whole hot path over one batch of synthetic
input: masked statistics sampling of N_s samples, the connected set and
amplitudes of every unique sample, E_loc with the count-weighted energy
statistics, and the VMC gradient.  Default workload: 7 spatial orbitals,
N_a = N_b = 5 (14 qubits, 441 determinants: the H2O shape of the paper's
Table I), synthetic integrals with 14 Cholesky vectors (seed 1), per-slot
MLP with 3 hidden layers of width 128, N_s = 1e5.

Prints one JSON line.  `value` = unique samples whose local energy was
completed, per second of device time (max over ranks), inputs resident in
HBM, L2 flushed between timed steps, for the chosen form (--form, default
BF16 tensor-core network); `forms` reports both forms timed the same way in
the same run (plain FP32 SIMT network and BF16), their ratio, and for each
the |E_gpu - E_oracle| of the count-weighted energy on that form's last
sample set against the FP64 oracle (evaluated in the CPU-baseline leg).  `e2e` = the same through the public
API with host buffers: parameters copied host->device and energy statistics
plus gradient copied back every step.  `--impl reference` times the FP64 CPU
oracle on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "local energies/sec at 1 GB300 (BF16 vs FP32 form), |dE| vs FP64 oracle (Ha)"
UNIT = "local energies/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """SM clocks and throttle reasons sampled during a region.

    NVML is read directly (libnvidia-ml through ctypes) every millisecond
    from a helper thread, so that even a timed region of a few milliseconds
    holds samples; nvidia-smi at its 20 ms period is the fallback when the
    library cannot be loaded.  Only reads: no setting of the GPU is changed."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.samples = []  # (time, sm_mhz, max_mhz, reason bits) from NVML
        self.nvml = None
        self.stop = threading.Event()
        self.source = "none"

    def _nvml_handle(self):
        import ctypes as C
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        h = C.c_void_p()
        # the CUDA device's own UUID first (NVML ignores CUDA_VISIBLE_DEVICES)
        try:
            u = str(torch.cuda.get_device_properties(self.index).uuid)
        except Exception:
            u = ""
        for cand in ([u, "GPU-" + u] if u else []):
            if lib.nvmlDeviceGetHandleByUUID(cand.encode(), C.byref(h)) == 0:
                return lib, h
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [s.strip() for s in vis.split(",") if s.strip()]
        idx = self.index
        if self.index < len(ids):
            if ids[self.index].isdigit():
                idx = int(ids[self.index])
            elif lib.nvmlDeviceGetHandleByUUID(ids[self.index].encode(), C.byref(h)) == 0:
                return lib, h
        if lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(idx), C.byref(h)) == 0:
            return lib, h
        return None

    def _poll(self):
        import ctypes as C
        lib, h = self.nvml
        mhz, mx, bits = C.c_uint(), C.c_uint(), C.c_ulonglong()
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop.is_set():
            if (lib.nvmlDeviceGetClockInfo(h, 1, C.byref(mhz)) == 0 and
                    lib.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx)) == 0 and get_reasons(h, C.byref(bits)) == 0):
                self.samples.append((time.perf_counter(), float(mhz.value), float(mx.value), int(bits.value)))
            time.sleep(0.001)

    def __enter__(self):
        try:
            self.nvml = self._nvml_handle()
        except OSError:
            self.nvml = None
        if self.nvml:
            self.source = "nvml 1 ms"
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
            t0 = time.perf_counter()
            while not self.samples and time.perf_counter() - t0 < 2.0:
                time.sleep(0.001)
        else:
            try:
                self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                              "--format=csv,noheader,nounits", "-lms", "20"],
                                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.source = "nvidia-smi 20 ms"
                self.t = threading.Thread(target=self._read, daemon=True)
                self.t.start()
                t0 = time.perf_counter()  # the sampler is running before the region starts
                while not self.lines and time.perf_counter() - t0 < 5.0:
                    time.sleep(0.01)
            except OSError:
                self.proc = None
        self.t_begin = time.perf_counter()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def __exit__(self, *a):
        self.t_end = time.perf_counter()
        self.stop.set()
        if self.nvml:
            self.t.join(timeout=1.0)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        if self.nvml:
            inside = [s for s in self.samples if self.t_begin <= s[0] <= self.t_end]
            for _, a, b, bits in inside:
                sm.append(a)
                mx.append(b)
                for bit, nm in self.REASONS.items():
                    if bits & bit:
                        reasons.add(nm)
        else:
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            inside = [ln for t, ln in self.lines if self.t_begin <= t <= self.t_end]
            if not inside:  # region shorter than the sampling period: the first sample after its start
                inside = [ln for t, ln in self.lines if t >= self.t_begin][:1]
            for ln in inside:
                f = [t.strip() for t in ln.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, f[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0,
                    "source": self.source}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "source": self.source}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if "WORLD_SIZE" in os.environ and "MASTER_ADDR" in os.environ:  # launched by torchrun
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        return ws, rank, local, dist
    return 1, 0, 0, None


def _cpu_baseline(w, sets=None, seconds=10.0, n_max=100000):
    """Time the FP64 oracle's local energy on the host cores.

    With ``sets`` ({form: {"x", "cnt", "stats"}}: the unique samples, counts
    and GPU statistics of a form's last timed step) the oracle evaluates
    those samples, a whole set when it fits in ``seconds`` per set, and
    reports |E_gpu - E_oracle| of the count-weighted energy on the same
    samples; otherwise it cycles over the unique samples of one oracle
    sampling pass.  The value is unique samples per second over all the
    oracle's work."""
    from oracle.anqs import MLPAnsatz, NADEAnsatz, TFAnsatz
    from oracle.hamiltonian import Hamiltonian as OHam
    from oracle.sampler import sample as osample
    from oracle.sector import molecular_isphys
    from oracle.vmc import energy_stats, local_energy

    oham = OHam(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    ip = molecular_isphys(w["n"], w["n_alpha"], w["n_beta"])
    if w["kind"] == "mlp":
        om = MLPAnsatz(w["params_struct"], w["n"])
    elif w["kind"] == "nade":
        om = NADEAnsatz(w["params_struct"], w["n"], ip)
    else:
        om = TFAnsatz(w["params_struct"], w["n"], w["n_heads"])
    k = 8
    if sets:
        done, busy, delta, notes = 0, 0.0, {}, []
        for form, st in sets.items():
            xs = st["x"].cpu().numpy().astype(np.uint64)
            es, t0 = [], time.perf_counter()
            for a in range(0, len(xs), k):
                if time.perf_counter() - t0 > seconds or done >= n_max:
                    break
                es.append(local_energy(om, ip, oham, xs[a:a + k]))
            dt = time.perf_counter() - t0
            m = sum(len(e) for e in es)
            done, busy = done + m, busy + dt
            notes.append(f"{m} of the {len(xs)} unique samples of the {form} form's last step")
            if m == len(xs):
                ref = energy_stats(np.concatenate(es), st["cnt"])
                delta[form] = {"E_oracle_ha": float(ref[0]), "abs_dE_ha": abs(float(st["stats"][0]) - ref[0]),
                               "_e_ref": np.concatenate(es)}
            else:
                delta[form] = {"abs_dE_ha": None, "note": "oracle did not finish the set in the time bound"}
        return {"value": done / busy, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                "sample": "FP64 oracle local energy (connected set + log psi + sum) of " + "; ".join(notes) +
                          f", {busy:.1f} s", "delta_E": delta}
    xs, _, _ = osample(om, ip, w["n"], w["n_samples"], seed=12345)
    done, t0 = 0, time.perf_counter()
    while done < n_max and time.perf_counter() - t0 < seconds:
        start = done % len(xs)
        chunk = xs[start:start + k]
        local_energy(om, ip, oham, chunk)
        done += len(chunk)
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle local energy (connected set + log psi + sum) of {done} unique samples "
                      f"(cycling over the {len(xs)} of one N_s={w['n_samples']} sampling pass), {dt:.1f} s"}


def _reference_arm(args, w, ws, rank):
    if rank != 0:
        return
    steps = []
    for _ in range(args.warmup):
        _cpu_baseline(w, seconds=2.0, n_max=16)
    for _ in range(args.steps):
        steps.append(_cpu_baseline(w, seconds=8.0, n_max=200))
    val = statistics.mean(s["value"] for s in steps)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / val,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(w, args),
            "cpu_baseline": {"kind": "oracle", "cores": steps[0]["cores"], "sample": steps[0]["sample"],
                             "value": val, "unit": UNIT},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(w, args):
    net = {"mlp": lambda: f"per-slot MLP {w['n_hidden']}x{w['width']}",
           "nade": lambda: f"per-qubit complex NADE (App. B.1) width {w['width']}",
           "tf": lambda: f"transformer d{w['d_model']} h{w['n_heads']} L{w['n_layers']}"}[w["kind"]]()
    return {"workload": f"{args.workload}: n_orb={w['n']} N_a={w['n_alpha']} N_b={w['n_beta']} "
                        f"({2 * w['n']} qubits), {w['n_chol']} Cholesky vectors seed {w['seed']}, {net}, "
                        f"N_s={args.n_samples or w['n_samples']}",
            "form": args.form, "n_samples": args.n_samples or w["n_samples"],
            "sampler": "binomial (chained binomials per node)" if args.binomial else "multinomial (one draw per sample)",
            "l2": "flushed between timed steps (256 MiB write)",
            "timing": "one CUDA-graph replay of the whole step per timed iteration (weight packing, sampling, "
                      "connected set, amplitudes, E_loc and statistics, gradient), CUDA events on the replay stream",
            "parallelism": (f"dp{args.gpus}: per-rank sample sets (seed per rank), statistics all-gather + "
                            "gradient all-reduce per step" if args.gpus > 1 else "single GPU")}


# DRAM bytes per launch from ncu captures of the same kernel build and
# workload (h2o, 16-bit form): dram__bytes_read.sum + dram__bytes_write.sum,
# each from the third step's launch of
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none
#       -k regex:<kernels> -s <2 steps of them> -c <1 step of them> --csv
#       python bench.py --steps 2 --warmup 3 --no-cpu-baseline --one-form --no-extra
# (the suffix with regex 'mlp_tc_ws|eloc_assemble|js_hist'; the slot launches,
# connected set, assembly and partial sum with
# 'connected_diag|mlp_tc_slots|eloc_assemble|partial_sum'); the adjoint from
# `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
# --clock-control none -c 80 --csv python bench.py --kernel-case`.  A kernel
# changed since its capture has no entry (traffic null).
TRAFFIC = {("h2o", "bf16"): {"mlp_tc_suffix_kernel": 1327104, "mlp_tc_parent_kernel": 660480,
                             "mlp_tc_slot_kernel": 663808, "mlp_tc_grad_kernel": 609792,
                             "eloc_assemble_kernel": 4674560, "connected_kernel": 64512,
                             "grad_partial_sum_kernel": 4014336}}


# kernel families that evaluate the connected determinants' amplitudes, in
# order of preference for the headline roofline
AMPLITUDE_FAMILIES = ("mlp_tc_suffix_kernel", "tf_tc_suffix_kernel", "nade_suffix_kernel", "tf_fp32_kernel")


def _make_model(A, w, params, form):
    if w["kind"] == "mlp":
        return A.Model.mlp(w["n"], w["width"], w["n_hidden"], params, form=form)
    if w["kind"] == "nade":
        return A.Model.nade(w["n"], w["width"], params)
    return A.Model.transformer(w["n"], w["d_model"], w["n_heads"], w["n_layers"], params, form=form)


def _run_form(A, lib, args, w, form, ham, params, dev, rank, dist, stream_clocks):
    """Graph-captured timing of one form: returns throughput, end-to-end
    throughput, the eager per-kernel profile and the last step's sample set
    with its statistics."""
    import ctypes as C
    model = _make_model(A, w, params, form)
    Ns = args.n_samples or w["n_samples"]
    cap = min(Ns, ham.sector_dim)
    i64, f64 = dict(dtype=torch.int64, device=dev), dict(dtype=torch.float64, device=dev)
    x, cnt, nu, ctr = torch.empty(cap, **i64), torch.empty(cap, **i64), torch.zeros(1, **i64), torch.zeros(1, **i64)
    ws_s = A._ws(A.sample_workspace_bytes(model, ham, Ns), dev)
    ws_e = A._ws(A.local_energy_workspace_bytes(model, ham, cap), dev)
    ws_g = A._ws(A.grad_workspace_bytes(model, ham, cap), dev)
    ere, eim, stats, stats_g = torch.zeros(cap, **f64), torch.zeros(cap, **f64), torch.zeros(4, **f64), \
        torch.zeros(4, **f64)
    g = torch.zeros(model.n_params, dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    seed = 1234 + 7919 * rank

    def step_a():
        if form == "bf16":
            model.sync()  # re-pack the bf16 weight images (the optimiser changes params every step)
        A.sample_into(model, ham, Ns, seed, 0, x, cnt, nu, ws_s, counter_dev=ctr, binomial=args.binomial)
        A.local_energy(model, ham, x, cnt, workspace=ws_e, n_dev=nu, out=(ere, eim, stats))

    def step_b(st):
        A.grad(model, ham, x, cnt, ere, eim, st, workspace=ws_g, n_dev=nu, out=g)
        ctr.add_(1)

    def step():
        """One pass of the hot path; every size stays on the device (the
        unique count of the sampler feeds the energy and gradient calls), so
        the pass can be captured in a CUDA graph and replayed.  The Philox
        counter advances on the device after each pass."""
        step_a()
        step_b(stats)

    def exchange():
        """Data-parallel exchange (one process per GPU, each with its own
        sample set): gather the ranks' statistics and combine them on the
        device; the gradients are summed after the gradient pass."""
        from paper_2310_04166_gb300.dist import exchange_stats
        A.stats_combine(exchange_stats(stats), out=stats_g)

    # eager warm-up, then a profiled eager pass (per-kernel CUDA-event times)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    lib.anqs_profile_enable(1)
    n_prof = max(5, min(args.steps // 2, 200))
    for _ in range(n_prof):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    prof = {}
    for pid in range(64):
        nm, n_l, ms = C.c_char_p(), C.c_uint64(), C.c_double()
        if lib.anqs_profile_read(pid, C.byref(nm), C.byref(n_l), C.byref(ms)) != 0:
            break
        if n_l.value:
            prof[nm.value.decode()] = (n_l.value, ms.value)
    lib.anqs_profile_enable(0)

    # capture the step in a CUDA graph
    l0 = C.c_uint64()
    lib.anqs_launch_count(C.byref(l0))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    l1 = C.c_uint64()
    lib.anqs_launch_count(C.byref(l1))
    launches_per_step = int(l1.value - l0.value)
    if dist:
        # two graphs around the exchange (the collectives run eagerly)
        from paper_2310_04166_gb300.dist import reduce_grad
        ga, gb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(ga):
            step_a()
        with torch.cuda.graph(gb):
            step_b(stats_g)

        class _Pair:
            def replay(self):
                ga.replay()
                exchange()
                gb.replay()
                reduce_grad(g)
        graph = _Pair()
    else:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()

    times, uniq = [], []
    stream = torch.cuda.current_stream()
    with Clocks(torch.cuda.current_device()) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            graph.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            uniq.append(int(nu.item()))
    if dist:
        dist.barrier()
    total_ms, total_u = sum(times), sum(uniq)
    if dist:
        t = torch.tensor([total_ms, float(total_u)], dtype=torch.float64, device=dev)
        tm = t.clone()
        dist.all_reduce(tm[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:], op=dist.ReduceOp.SUM)
        total_ms, total_u = float(tm[0]), float(t[1])
    value = total_u / (total_ms / 1e3)
    k_last = int(nu.item())
    last = {"x": x[:k_last].clone(), "cnt": cnt[:k_last].cpu().numpy(), "stats": stats.cpu().numpy().copy(),
            "ere": ere[:k_last].cpu().numpy().copy()}

    # end to end through the public API: host parameters in, host energy
    # statistics and gradient out, around each graph replay
    h_params = params.detach().cpu().pin_memory()
    h_stats = torch.empty(4, dtype=torch.float64).pin_memory()
    h_grad = torch.empty(model.n_params, dtype=torch.float32).pin_memory()
    e2e_ms, e2e_u = 0.0, 0
    for i in range(max(3, args.steps)):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        params.copy_(h_params, non_blocking=True)
        graph.replay()
        h_stats.copy_(stats_g if dist else stats, non_blocking=True)
        h_grad.copy_(g, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_u += int(nu.item())
    return {"model": model, "value": value, "ms_per_step": total_ms / args.steps, "n_unique": total_u / args.steps,
            "e2e": {"value": e2e_u / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(params.numel() * 4),
                    "d2h_bytes_per_step": int(4 * 8 + model.n_params * 4 + 8)},
            "launches_per_step": launches_per_step, "prof": prof, "n_prof": n_prof, "last": last,
            "clocks": clk.summary()}


def _oracle_model(w):
    from oracle.anqs import MLPAnsatz, TFAnsatz
    from oracle.sector import molecular_isphys
    ip = molecular_isphys(w["n"], w["n_alpha"], w["n_beta"])
    om = MLPAnsatz(w["params_struct"], w["n"]) if w["kind"] == "mlp" else TFAnsatz(w["params_struct"], w["n"],
                                                                                    w["n_heads"])
    return om, ip


def _grad_vs_oracle(A, model, ham, w, x, cnt, e_ref):
    """Relative L2 distance between the form's VMC gradient (Eq. grad_def) on
    the samples x with counts cnt (its own local energies and statistics, all
    through the library) and the FP64 oracle's gradient on the same samples
    from the oracle's local energies e_ref."""
    from oracle.vmc import energy_stats, gradient
    om, ip = _oracle_model(w)
    c = torch.as_tensor(np.asarray(cnt, dtype=np.int64), device=x.device)
    ere, eim, st = A.local_energy(model, ham, x, c)
    g = A.grad(model, ham, x, c, ere, eim, st).cpu().numpy().astype(np.float64)
    xs = x.cpu().numpy().astype(np.uint64)
    s_ref = energy_stats(e_ref, cnt)
    g_ref = np.concatenate([t.reshape(-1).numpy() for t in gradient(om, ip, xs, cnt, e_ref, s_ref)])
    return float(np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref))


def _oracle_subset(w, last, m=48, seed=7, A=None, model=None, ham=None):
    """|E_gpu - E_oracle| estimated from m samples of the step's unique set,
    drawn with probability proportional to their counts: the mean of
    E_loc,gpu - E_loc,oracle over the draws is an unbiased estimate of the
    count-weighted energy difference (its standard error beside it).  For
    sample sets too large for the FP64 oracle to evaluate whole within the
    bench's time bound."""
    from oracle.hamiltonian import Hamiltonian as OHam
    from oracle.vmc import local_energy
    oham = OHam(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    om, ip = _oracle_model(w)
    xs = last["x"].cpu().numpy().astype(np.uint64)
    cnt = np.asarray(last["cnt"], dtype=np.float64)
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(xs), size=min(m, len(xs)), replace=True, p=cnt / cnt.sum())
    uniq, inv = np.unique(pick, return_inverse=True)
    t0 = time.perf_counter()
    e_c = np.concatenate([local_energy(om, ip, oham, xs[uniq[a:a + 8]]) for a in range(0, len(uniq), 8)])
    d = (last["ere"][uniq] - e_c.real)[inv]
    out = {"abs_dE_ha_estimate": abs(float(d.mean())), "stderr_ha": float(d.std(ddof=1) / np.sqrt(len(d))),
           "max_abs_dEloc_ha": float(np.abs(d).max()), "draws": int(len(d)), "oracle_s": time.perf_counter() - t0,
           "how": f"{len(d)} draws (proportional to counts) of the {len(xs)} unique samples, FP64 oracle E_loc"}
    if A is not None:  # the gradient restricted to the drawn samples (their counts in the step's set)
        sel = torch.as_tensor(uniq, device=last["x"].device)
        out["grad_rel_l2"] = _grad_vs_oracle(A, model, ham, w, last["x"][sel].contiguous(), cnt[uniq], e_c)
        out["grad_how"] = (f"gradient on the {len(uniq)} distinct drawn samples with their step counts: library "
                           "(own local energies) against the FP64 oracle")
    return out


def _sub_workload(A, lib, args, name, dev, rank, dist, steps):
    """Both forms of another workload, timed as the headline one (graph replay
    of the whole step, L2 flushed between steps), with the amplitude
    contraction's roofline and the oracle comparison on a count-weighted
    subset of each form's last sample set."""
    import copy
    from synthetic import workload
    w = workload(name)
    a = copy.copy(args)
    a.steps, a.n_samples, a.binomial, a.workload = steps, 0, False, name
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    params = torch.tensor(w["params"], device=dev)
    out = {"config": _config(w, a)["workload"], "steps": steps}
    peaks, src = _peaks()
    for form in ("bf16", "fp32"):
        r = _run_form(A, lib, a, w, form, ham, params, dev, rank, dist, True)
        work = _tc_work(A, ham, r["model"], w, r["last"]["x"])
        roof, _ = _rooflines(r["prof"], work, r["n_prof"], peaks, src, {})
        f = {"value": r["value"], "ms_per_step": r["ms_per_step"], "n_unique_per_step": r["n_unique"],
             "E_ha": float(r["last"]["stats"][0]), "clocks": r["clocks"]}
        if roof:
            f["roofline"] = {k: roof[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac",
                                                  "avg_launch_us")}
        if not args.no_cpu_baseline:  # more draws for the 16-bit form, whose per-sample deviations are larger
            f["oracle"] = _oracle_subset(w, r["last"], m=256 if form == "bf16" else 64, A=A, model=r["model"],
                                         ham=ham)
        out[form] = f
        del r
        torch.cuda.empty_cache()
    out["bf16_over_fp32"] = out["bf16"]["value"] / out["fp32"]["value"]
    return out


def _large(args, dev, quick=False):
    """Config-4 shape (26 orbitals, 9+9 electrons, transformer d128 h8 L4,
    33,507 connected determinants per sample): local energies per second of
    anqs_local_energy over a bounded sample (the 64 most frequent unique
    samples of one 2000-sample pass), BF16 tensor-core form (keys and values
    of the parent reused) against the plain FP32 form on the same samples,
    with the amplitude kernel's roofline and the BF16 form's local-energy
    deviation from the FP32 form (which is checked against its FP64 definition
    at this shape).  An auxiliary line, not the headline workload."""
    import ctypes as C
    import paper_2310_04166_gb300 as A
    from paper_2310_04166_gb300 import _lib
    from synthetic import workload
    lib = _lib.load()
    w = workload("large")
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    params = torch.tensor(w["params"], device=dev)
    models = {f: A.Model.transformer(w["n"], w["d_model"], w["n_heads"], w["n_layers"], params, form=f)
              for f in ("bf16", "fp32")}
    x, c = A.sample(models["fp32"], ham, 2000, seed=1234)
    keep = torch.argsort(c, descending=True, stable=True)[:64]
    x, c = x[keep].contiguous(), c[keep].contiguous()
    ws = A._ws(max(A.local_energy_workspace_bytes(m, ham, x.numel()) for m in models.values()), dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    res, outs = {}, {}
    peaks, src = _peaks()
    for form, model in models.items():
        out = (torch.empty(x.numel(), dtype=torch.float64, device=dev),
               torch.empty(x.numel(), dtype=torch.float64, device=dev), torch.empty(4, dtype=torch.float64, device=dev))
        steps = (min(args.steps, 3) if quick else args.steps) if form == "bf16" else max(1, min(args.steps, 1 if quick else 2))
        for _ in range(args.warmup if form == "bf16" else 1):
            A.local_energy(model, ham, x, c, workspace=ws, out=out)
        torch.cuda.synchronize()
        lib.anqs_profile_enable(1)
        A.local_energy(model, ham, x, c, workspace=ws, out=out)
        torch.cuda.synchronize()
        prof = {}
        for pid in range(64):
            nm, n_l, ms = C.c_char_p(), C.c_uint64(), C.c_double()
            if lib.anqs_profile_read(pid, C.byref(nm), C.byref(n_l), C.byref(ms)) != 0:
                break
            if n_l.value:
                prof[nm.value.decode()] = (n_l.value, ms.value)
        lib.anqs_profile_enable(0)
        stream = torch.cuda.current_stream()
        times = []
        with Clocks(dev.index or 0) as clk:
            for i in range(steps):
                flush.fill_(i & 0xFF)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                A.local_energy(model, ham, x, c, workspace=ws, out=out)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
        ms = sum(times) / len(times)
        work = _tf_work(A, ham, w, x)
        roof, _ = _rooflines(prof, work, 1, peaks, src, {})
        res[form] = {"value": x.numel() / (ms / 1e3), "ms_per_step": ms, "steps": steps, "clocks": clk.summary(),
                     "roofline": roof, "status": model.status()}
        outs[form] = (out[0].clone(), out[2].clone())
    d = (outs["bf16"][0] - outs["fp32"][0]).abs()
    K = ham.n_connected
    r = res["bf16"]
    return ({"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": r["steps"],
                      "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "fp16-operand tcgen05 GEMM (kind::f16, f32 accumulate) / f32 heads / f64 E_loc",
                      "data": "synthetic",
                      "config": {"workload": f"large: n_orb={w['n']} N_a={w['n_alpha']} N_b={w['n_beta']}, "
                                             f"transformer d{w['d_model']} h{w['n_heads']} L{w['n_layers']}, "
                                             f"{x.numel()} unique samples x {K} connected determinants per step",
                                 "timed": "anqs_local_energy only (connected set, amplitudes, E_loc, statistics)",
                                 "l2": f"flushed between timed steps; working set above L2 ({x.numel() * K} "
                                       "connected determinants)"},
                      "roofline": r["roofline"], "clocks": r["clocks"],
                      "forms": {"bf16": res["bf16"], "fp32": res["fp32"],
                                "bf16_over_fp32": res["bf16"]["value"] / res["fp32"]["value"],
                                "bf16_vs_fp32": {"max_abs_dEloc_ha": float(d.max()),
                                                 "abs_dE_ha": abs(float(outs["bf16"][1][0] - outs["fp32"][1][0])),
                                                 "note": "FP32 form = E_loc definition within 1e-6 relative "
                                                         "(tests/test_gpu_tf.py)"}}})


def _batch32(args, dev, quick=False):
    """32 independent problems (seeds 100..131, n in [6, 14], MLP 3x128 each,
    N_s = 1e5 each), every arm one CUDA-graph replay of all 32 passes
    (sampling, local energies, gradient) per timed step:
      16-bit persistent: samplers and gradients on one stream per problem,
        the local energies in one batched call whose amplitude stage is one
        persistent launch over every (problem, slot, tile), schedule chosen
        by the library's autotuner (the headline of this line);
      16-bit streams: every problem's whole pass on its own stream;
      FP32 streams: the plain form, scheduled the same way;
    plus the plain form as 32 eager passes one after the other.  The oracle
    checks |E_gpu - E_oracle| on the problems whose unique sets it finishes
    quickly.  Prints one JSON line."""
    import paper_2310_04166_gb300 as A
    from paper_2310_04166_gb300 import _lib
    from paper_2310_04166_gb300.batch import BatchedStep, Problem
    from synthetic import batch32_problem, flatten_mlp, mlp_params
    specs = [batch32_problem(k) for k in range(32)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    steps = max(1, min(args.steps, 3 if quick else 20))

    def build(form):
        out = []
        for k, p in enumerate(specs):
            ham = A.Hamiltonian(p["h"], p["g"], p["e_nuc"], p["n_alpha"], p["n_beta"])
            params = torch.tensor(flatten_mlp(mlp_params(p["seed"], p["n"], p["width"], p["n_hidden"])), device=dev)
            model = A.Model.mlp(p["n"], p["width"], p["n_hidden"], params, form=form)
            out.append(Problem(ham, model, p["n_samples"], 1234 + k))
        return out

    def timed(run, problems, n):
        times, uniq = [], 0
        stream = torch.cuda.current_stream()
        for i in range(n):
            flush.fill_(i & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            run()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            uniq += int(torch.stack([p.nu for p in problems]).sum().item())
        return {"value": uniq / (sum(times) / 1e3), "ms_per_step": sum(times) / n, "n_unique_per_step": uniq / n}

    def graph_arm(form, persistent):
        # the FP32 arms take about 13 s a step: one warm-up pass and 3 timed steps (1 in the quick form)
        warm, n_timed = (args.warmup, steps) if form == "bf16" else (1, 1 if quick else max(1, min(steps, 3)))
        probs = build(form)
        bs = BatchedStep(probs, persistent=persistent)
        for _ in range(warm):
            bs.eager()
        extra = {}
        if persistent:
            t = bs.autotune()
            mode, chunk = bs.energy.schedule
            names = ["static" if m == _lib.ANQS_BATCH_STATIC else f"dynamic_chunk{c}"
                     for m, c in A.AUTOTUNE_CANDIDATES]
            extra["autotuner"] = {"times_ms": {nm: round(v, 4) for nm, v in zip(names, t)},
                                  "chosen": {"mode": "static" if mode == _lib.ANQS_BATCH_STATIC else "dynamic",
                                             "chunk": chunk}}
            # roofline of the persistent amplitude launch: the suffix FLOP (with prefix
            # reuse) of the sample sets the autotuner timed, over its fastest time
            flop = 0.0
            for sp, pr in zip(specs, probs):
                nu = int(pr.nu.item())
                flop += _tc_work(A, pr.ham, pr.model, sp, pr.x[:nu].contiguous())["mlp_tc_suffix_kernel"]
            peaks, src = _peaks()
            best = min(t)
            ach = flop / (best / 1e3) / 1e12
            extra["roofline"] = {"kernel": "mlp_tc_multi_kernel", "bound": "tensor", "achieved": ach,
                                 "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "frac": ach / peaks["bf16_tflops"],
                                 "traffic": None, "avg_launch_us": best * 1e3, "work_per_launch": flop,
                                 "note": f"dense bf16 {src} burst peak; suffix FLOP with prefix reuse of the 32 "
                                         "problems over the autotuner's fastest launch time"}
        bs.capture()
        for _ in range(warm):
            bs.replay()
        with Clocks(torch.cuda.current_device()) as clk:
            r = timed(bs.replay, probs, n_timed)
        r["steps"] = n_timed
        r.update(extra)
        r["clocks"] = clk.summary()
        return r, probs

    res = {}
    res["bf16_persistent"], probs = graph_arm("bf16", True)
    oracle = None if args.no_cpu_baseline else _batch32_oracle(specs, probs, 10.0 if quick else 20.0)
    del probs
    torch.cuda.empty_cache()
    res["bf16_streams"], probs = graph_arm("bf16", False)
    del probs
    torch.cuda.empty_cache()
    res["fp32_streams"], probs = graph_arm("fp32", False)

    def plain():
        for p in probs:
            p.step()
    if not quick:  # 32 eager FP32 passes (left out of the default line: the graph arm above times the same work)
        plain()
        res["fp32_separate"] = timed(plain, probs, max(1, min(steps, 3)))
    head = res["bf16_persistent"]
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp16-operand tcgen05 GEMM (kind::f16, f32 accumulate) / f32 heads / f64 E_loc",
            "data": "synthetic",
            "config": {"workload": "batch32: 32 problems, seeds 100..131, n in [6, 14], N_a = N_b in [1, n-1], "
                                   "2n Cholesky vectors, per-slot MLP 3x128 each, N_s = 1e5 each",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "timing": "one CUDA-graph replay of all 32 passes per timed step (weight packing, sampling, "
                                 "local energies and statistics, gradient); fp32_separate: 32 eager passes one "
                                 "after the other"},
            "n_unique_per_step": head["n_unique_per_step"],
            "roofline": head.get("roofline"),
            "forms": dict(res, bf16_persistent_over_fp32_streams=head["value"] / res["fp32_streams"]["value"],
                          bf16_persistent_over_bf16_streams=head["value"] / res["bf16_streams"]["value"],
                          **({"bf16_persistent_over_fp32_separate": head["value"] / res["fp32_separate"]["value"]}
                             if "fp32_separate" in res else {})),
            "clocks": head["clocks"]}
    if oracle:
        line["oracle"] = oracle
    return line


def _batch32_oracle(specs, probs, seconds=20.0):
    """|E_gpu - E_oracle| of the 16-bit persistent arm's last step, per
    problem, for the problems whose whole unique set the FP64 oracle
    evaluates within the time bound (smallest sets first)."""
    from oracle.anqs import MLPAnsatz
    from oracle.hamiltonian import Hamiltonian as OHam
    from oracle.sector import molecular_isphys
    from oracle.vmc import energy_stats, local_energy
    from synthetic import mlp_params
    order = sorted(range(len(probs)), key=lambda k: int(probs[k].nu.item()) * probs[k].ham.n_connected)
    out, t0 = {}, time.perf_counter()
    for k in order:
        if time.perf_counter() - t0 > seconds:
            break
        sp, pr = specs[k], probs[k]
        nu = int(pr.nu.item())
        xs = pr.x[:nu].cpu().numpy().astype(np.uint64)
        cnt = pr.cnt[:nu].cpu().numpy()
        oham = OHam(sp["h"], sp["g"], sp["e_nuc"], sp["n_alpha"], sp["n_beta"])
        ip = molecular_isphys(sp["n"], sp["n_alpha"], sp["n_beta"])
        om = MLPAnsatz(mlp_params(sp["seed"], sp["n"], sp["width"], sp["n_hidden"]), sp["n"])
        e = np.concatenate([local_energy(om, ip, oham, xs[a:a + 8]) for a in range(0, nu, 8)])
        ref = energy_stats(e, cnt)
        out[f"problem{k}"] = {"n": sp["n"], "n_alpha": sp["n_alpha"], "unique": nu,
                              "abs_dE_ha": abs(float(pr.stats[0].item()) - float(ref[0]))}
    return {"per_problem": out, "how": f"FP64 oracle local energy of each problem's whole unique set, smallest "
                                       f"sets first, within {seconds:.0f} s"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default=os.environ.get("ANQS_BENCH_FORM", "bf16"), choices=["fp32", "bf16"])
    ap.add_argument("--workload", default="h2o")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--one-form", action="store_true", help="time only --form (default: both forms)")
    ap.add_argument("--no-extra", action="store_true", help="h2o only: leave out the n2, batch32 and large sub-workloads")
    ap.add_argument("--binomial", action="store_true", help="binomial statistics sampling (chained binomials per node)")
    ap.add_argument("--n-samples", type=float, default=0, help="N_s of the sampling pass (default: the workload's)")
    ap.add_argument("--kernel-samples", type=int, default=0,
                    help="--kernel-case: keep only the K most frequent samples and leave out the gradient call")
    ap.add_argument("--kernel-case", action="store_true",
                    help="one FP32-form sampling pass, then one local-energy and one gradient call in the "
                         "chosen form (the launch sequence to capture with ncu), then exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    args.n_samples = int(args.n_samples)

    from synthetic import workload
    w = workload("h2o" if args.workload == "batch32" else args.workload)
    ws, rank, local, dist = _dist()
    if args.impl == "reference":
        _reference_arm(args, w, ws, rank)
        if dist:
            dist.destroy_process_group()
        return

    import paper_2310_04166_gb300 as A
    from paper_2310_04166_gb300 import _lib
    lib = _lib.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.workload == "batch32":
        print(json.dumps(_batch32(args, dev)), flush=True)
        return
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    params = torch.tensor(w["params"], device=dev)
    if w["kind"] == "nade":  # the NADE has the FP32 form only
        args.form, args.one_form = "fp32", True
    form = args.form
    if args.workload == "large" and not args.kernel_case:
        print(json.dumps(_large(args, dev)), flush=True)
        return
    if args.kernel_case:
        model = _make_model(A, w, params, form)
        m32 = _make_model(A, w, params, "fp32")
        xk, nk = A.sample(m32, ham, w.get("n_samples", 2000), seed=99)
        if args.kernel_samples:  # the most frequent few (a small case of the same kernels)
            keep = torch.argsort(nk, descending=True, stable=True)[:args.kernel_samples]
            xk, nk = xk[keep].contiguous(), nk[keep].contiguous()
        ek = A.local_energy(model, ham, xk, nk)
        if not args.kernel_samples:
            A.grad(model, ham, xk, nk, ek[0], ek[1], ek[2])
        torch.cuda.synchronize()
        print(json.dumps({"kernel_case": args.workload, "form": form, "n_unique": xk.numel(),
                          "E": float(ek[2][0])}))
        return

    runs = {form: _run_form(A, lib, args, w, form, ham, params, dev, rank, dist, True)}
    if not args.one_form:
        other = "fp32" if form == "bf16" else "bf16"
        runs[other] = _run_form(A, lib, args, w, other, ham, params, dev, rank, dist, True)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    r = runs[form]

    # rooflines of the kernel families (eager profiled pass)
    peaks, src = _peaks()
    work = _tc_work(A, ham, r["model"], w, r["last"]["x"])
    roof, roofs = _rooflines(r["prof"], work, r["n_prof"], peaks, src, TRAFFIC.get((args.workload, form), {}))
    top = max(r["prof"].items(), key=lambda kv: kv[1][1])[0] if r["prof"] else None

    cpu = None
    if not args.no_cpu_baseline:
        cpu = _cpu_baseline(w, {f: v["last"] for f, v in runs.items()})
    forms = {f: {"value": v["value"], "ms_per_step": v["ms_per_step"], "e2e": v["e2e"]["value"],
                 "n_unique_per_step": v["n_unique"], "E_ha": float(v["last"]["stats"][0])} for f, v in runs.items()}
    if cpu:
        for f, d in cpu.pop("delta_E", {}).items():
            e_ref = d.pop("_e_ref", None)
            forms[f].update(d)
            if e_ref is not None:  # the whole set evaluated by the oracle: the gradient on it too
                v = runs[f]
                forms[f]["grad_rel_l2"] = _grad_vs_oracle(A, v["model"], ham, w, v["last"]["x"], v["last"]["cnt"],
                                                          e_ref)
    if "fp32" in runs and "bf16" in runs:
        forms["bf16_over_fp32"] = runs["bf16"]["value"] / runs["fp32"]["value"]
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "fp16-operand tcgen05 GEMM (kind::f16, f32 accumulate) / f32 heads / f64 E_loc" if form == "bf16" else "f32 network / f64 E_loc",
            "data": "synthetic", "config": _config(w, args), "n_unique_per_step": r["n_unique"],
            "e2e": r["e2e"], "forms": forms,
            "gpu_launches": r["launches_per_step"] * args.steps,
            "launches_per_step": r["launches_per_step"],
            "kernels": {k: {"launches": v[0], "total_ms": round(v[1], 4)} for k, v in r["prof"].items()},
            "kernels_note": f"CUDA-event totals over {r['n_prof']} eager (non-graph) steps",
            "roofline": roof, "rooflines": roofs, "top_kernel_family": top, "clocks": r["clocks"]}
    if cpu:
        line["cpu_baseline"] = cpu
    if args.workload == "h2o" and not args.no_extra and ws == 1:
        # the N2-shaped transformer workload in the same line, fewer steps (its FP32 form takes ~0.75 s a step),
        # then the 32-problem batch (persistent launch, autotuned) and the 26-orbital transformer in short forms;
        # a sub-workload that fails records its error and the line still prints
        subs = (("n2", lambda: _sub_workload(A, lib, args, "n2", dev, rank, dist, min(args.steps, 10))),
                ("batch32", lambda: _compact(_batch32(args, dev, quick=True))),
                ("large", lambda: _compact(_large(args, dev, quick=True))))
        line["workloads"] = {}
        for name, run in subs:
            line["workloads"][name] = _guarded(run)
            _guarded(torch.cuda.empty_cache)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _guarded(run):
    """run(), or {"error": ...} if it raises: one sub-workload's failure
    must not take the headline line with it."""
    try:
        return run()
    except Exception as e:  # noqa: BLE001 (any failure of a sub-workload is reported, not raised)
        return {"error": f"{type(e).__name__}: {e}"[:400]}


def _compact(sub):
    """A workload's own line without the keys the enclosing line already has."""
    return {k: v for k, v in sub.items() if k not in ("metric", "unit", "n_gpus", "higher_is_better", "scaling",
                                                        "vs_baseline", "data")}


def _tf_work(A, ham, w, x):
    """Algorithmic FLOP per step of the transformer families for the sample
    set x.  One (sequence, position t) row costs f(t) = L (24 d^2 + 4 (t+1) d)
    + 16 d: the q|k|v, output and FFN projections, the attention scores and
    weighted sum over the t+1 keys, and the head.  suffix = positions > j(x')
    of every connected x'; parent = every position of every sample; slot
    (sampler) = positions 0..p of every distinct prefix at level p; grad =
    3 x parent (forward plus the two products of the adjoint)."""
    n, d, L = w["n"], w["d_model"], w["n_layers"]
    f = np.array([L * (24 * d * d + 4 * (t + 1) * d) + 16 * d for t in range(n)], dtype=np.float64)
    cf = np.concatenate([[0.0], np.cumsum(f)])
    xp, hv, js, hd = A.connected(ham, x)
    j = js.reshape(-1).cpu().numpy().astype(np.int64)
    suffix = float((cf[n] - cf[j + 1]).sum())
    parent = float(len(x) * cf[n])
    xs = x.cpu().numpy().astype(np.uint64)
    slot = 0.0
    for p in range(n):
        pre = np.unique(xs & np.uint64((1 << (2 * p)) - 1)) if p else np.zeros(1, np.uint64)
        slot += len(pre) * cf[p + 1]
    eloc_bytes = float((8 + 1 + 8 + 8 + 8 * (n - 1 - j)).sum())
    return {"tf_tc_suffix_kernel": suffix, "tf_tc_parent_kernel": parent, "tf_tc_slot_kernel": slot,
            "tf_fp32_kernel": len(j) * cf[n] + parent + slot, "tf_fp32_grad_kernels": 3.0 * parent,
            "eloc_assemble_kernel": eloc_bytes, "connected_kernel": float(len(j) * (8 + 8 + 1) + len(x) * 8)}


def _tc_work(A, ham, model, w, x):
    """Algorithmic work per step for the sample set x.

    FLOP of one slot-p evaluation f(p) = 2 (4p W + (L-1) W^2 + 8 W).
    suffix = sum over connected x' of f(p) for the slots p > j(x'); parent =
    every slot of every sample; slot (sampler) = every slot of every distinct
    prefix of the leaves (the frontier of each level); grad = 3 x parent (the
    forward recomputed plus the two adjoint products); eloc bytes = per
    connected x': x' 8 + j 1 + H 8 + parent cache 8 + one 8-byte term per
    slot p > j."""
    if w["kind"] == "nade":
        return _nade_work(A, ham, w, x)
    if w["kind"] != "mlp":
        return _tf_work(A, ham, w, x)
    n, W, L = w["n"], w["width"], w["n_hidden"]
    f = np.array([2 * (4 * p * W + (L - 1) * W * W + 8 * W) for p in range(n)], dtype=np.float64)
    cf = np.concatenate([[0.0], np.cumsum(f)])  # cf[p] = sum_{q<p} f[q]
    xp, hv, js, hd = A.connected(ham, x)
    j = js.reshape(-1).cpu().numpy().astype(np.int64)
    suffix = float((cf[n] - cf[j + 1]).sum())
    parent = float(len(x) * cf[n])
    xs = x.cpu().numpy().astype(np.uint64)
    slot = 0.0
    for p in range(n):
        pre = np.unique(xs & np.uint64((1 << (2 * p)) - 1)) if p else np.zeros(1, np.uint64)
        slot += len(pre) * f[p]
    eloc_bytes = float((8 + 1 + 8 + 8 + 8 * (n - 1 - j)).sum())
    return {"mlp_tc_suffix_kernel": suffix, "mlp_tc_parent_kernel": parent, "mlp_tc_slot_kernel": slot,
            "mlp_fp32_grad_kernel": 3.0 * parent, "mlp_tc_grad_kernel": 3.0 * parent, "eloc_assemble_kernel": eloc_bytes,
            "connected_kernel": float(len(j) * (8 + 8 + 1) + len(x) * 8)}


def _nade_work(A, ham, w, x):
    """Algorithmic FLOP per step of the NADE kernels for the sample set x.
    One evaluation of qubit i costs f(i) = 8 W^2 + 16 W + 2 i W (complex
    W2 h1 and W3 h2 at 8 FLOP per complex multiply-add, the W1 columns of
    the set bits counted as all i).  parent = the 8 values of every slot of
    every sample, f(2p) + 2 f(2p+1) per slot (qubit 2p+1 for both values of
    qubit 2p); suffix = the path qubits 2p, 2p+1 of the slots p > j(x') of
    every connected x'; slot (sampler) = slot p of every distinct prefix at
    level p; grad = 3 f(i) per (sample, qubit): the forward and the two
    adjoint products."""
    n, W = w["n"], w["width"]
    f = np.array([8 * W * W + 16 * W + 2 * i * W for i in range(2 * n)], dtype=np.float64)
    slot = f[0::2] + 2 * f[1::2]
    path = f[0::2] + f[1::2]
    cpath = np.concatenate([[0.0], np.cumsum(path)])  # cpath[p] = sum_{q<p} path[q]
    _, _, js, _ = A.connected(ham, x)
    j = js.reshape(-1).cpu().numpy().astype(np.int64)
    xs = x.cpu().numpy().astype(np.uint64)
    samp = 0.0
    for p in range(n):
        pre = np.unique(xs & np.uint64((1 << (2 * p)) - 1)) if p else np.zeros(1, np.uint64)
        samp += len(pre) * slot[p]
    return {"nade_parent_kernel": len(xs) * slot.sum(), "nade_suffix_kernel": float((cpath[n] - cpath[j + 1]).sum()),
            "nade_slot_kernel": samp, "nade_grad_kernel": 3.0 * len(xs) * f.sum()}


def _rooflines(prof, work, steps, peaks, src, traffic):
    """Roofline of every kernel family with a defined bound (work per step x
    steps / total event time) and the dominant one by time."""
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    out = {}
    for name, (launches, ms) in prof.items():
        if name not in work or ms <= 0:
            continue
        per_launch = work[name] * steps / launches
        avg_s = ms / launches * 1e-3
        if name.startswith(("mlp_tc_", "tf_tc_")):
            bound, unit, peak = "tensor", "TFLOP/s", peaks["bf16_tflops"]
            ach = per_launch / avg_s / 1e12
            note = f"dense bf16 {src} burst peak; FLOP with prefix reuse"
        elif name in ("mlp_fp32_grad_kernel", "tf_fp32_grad_kernels", "tf_fp32_kernel") or name.startswith("nade_"):
            bound, unit, peak = "alu", "TFLOP/s", fp32_peak
            ach = per_launch / avg_s / 1e12
            note = f"FP32 SIMT peak derived: 152 SMs x 128 FMA lanes x 2 x {sm_mhz:.0f} MHz"
        else:
            bound, unit, peak = "hbm", "GB/s", peaks["hbm_gbs"]
            ach = per_launch / avg_s / 1e9
            note = f"{src} copy bandwidth; algorithmic bytes"
        out[name] = {"kernel": name, "bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                     "frac": ach / peak, "traffic": traffic.get(name), "avg_launch_us": avg_s * 1e6,
                     "work_per_launch": per_launch, "note": note}
    # the headline is the amplitude contraction of the connected determinants
    # (the bulk of the tensor work); the other families stay under `rooflines`
    headline = next((out[k] for k in AMPLITUDE_FAMILIES if k in out), None)
    if headline is None and out:
        headline = max(out.values(), key=lambda r: prof[r["kernel"]][1])
    return headline, out


if __name__ == "__main__":
    main()
