#!/usr/bin/env python
"""Benchmark of the DPG hot path on B300: one step = one whole forward pass.

Step (all on the GPU, through libdpg's C ABI):
  element pass  - quadrature, G_K = L L^H, condensation to S_K, s_K (Sec. 2.3, Algorithm 2)
  assembly      - deterministic sum of S_K, s_K into the CSR trace system
  CG            - to relative residual 1e-10 (default: FP32-inner iterative refinement with
                  entity-block Jacobi preconditioning, the inner operator applied element by element
                  from FP32 tiles of S_K; --cg fp64 gives the paper's plain FP64 CG)
  estimate      - local recovery of u and the residual estimator eta_K
Metric: DPG elements per second of the whole step (inputs resident in HBM), with
the CG time-to-1e-10 and the per-phase breakdown in the same JSON line.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun, one rank per GPU): every rank solves its own replica
(weak scaling; the method's CG would need a halo exchange, not built here).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DPG elements/s (local solve+η_K) & CG time-to-1e-10; mixed/batched vs FP64"
UNIT = "elements/s"
CG_MODES = {"fp64": 0, "ir": 1, "fp64-jacobi": 2, "ir-jacobi": 3, "fp64-bjacobi": 4, "ir-bjacobi": 5,
            "ir-bjacobi-half": 5 | 16, "ir64v-bjacobi": 5 | 32, "ir64v": 1 | 32,
            "dw": 64, "dw-bjacobi": 64 | 4, "ir-ebe": 1 | 128, "ir-bjacobi-ebe": 5 | 128,
            "ir-bjacobi-rel": 5 | 256, "ir-bjacobi-ebe-rel": 5 | 128 | 256, "ir-bjacobi-ebe-bulk": 5 | 128 | 512}
PRECISIONS = {"fp64": 0, "tf32": 1, "3xtf32": 2}


def config_mesh(name):
    from paper_2609_03155_b300 import inputs
    if name == "waveguide3d":
        return inputs.waveguide_3d_config(32, 16, 64, 2)
    if name == "waveguide3d-small":
        return inputs.waveguide_3d_config(8, 4, 16, 2)
    if name == "waveguide3d-medium":
        return inputs.waveguide_3d_config(16, 8, 32, 2)
    if name == "waveguide3d-profile":
        # small enough for ncu captures (a few GB on the device), CSR larger than L2
        return inputs.waveguide_3d_config(12, 6, 24, 2)
    if name == "waveguide2d":
        return inputs.waveguide_2d_config(p=1)
    if name == "cavity3":
        # jittered unit cavity, p = 3, random lossy permittivity; 16^3 elements
        # (2^18 elements at p = 3 need ~1.3 TB of condensation data and CSR)
        return inputs.cavity(16, 3, jitter=0.1, eps_mode='random', name="cavity3_16x16x16_p3_jitter0.1")
    if name == "fichera":
        # Fichera-corner cavity, graded toward the re-entrant corner, degrees
        # 1..4 in a 40/30/20/10 % mix; 12 cells per unit length (13,824 elements)
        m = inputs.fichera_cavity(12, grade=1.5, name="fichera_12_graded_p1234")
        return m
    if name == "fichera-amr":
        # Fichera cavity, 12 coarse cells per unit, cells within 0.3 of the
        # re-entrant corner refined once (2:1 hanging faces), degrees 1..4 mixed
        return inputs.fichera_amr(12, radius=0.3)
    if name == "cavity3-32":
        # the 32^3 sub-box of the jittered p = 3 cavity with random lossy permittivity (2^18 elements at p = 3
        # need a CSR of ~661 GB; the element rate is the same per element)
        return inputs.cavity(32, 3, jitter=0.1, eps_mode='random', name="cavity3_32x32x32_p3_jitter0.1")
    if name == "fichera-amr-1e5":
        # Fichera cavity, 20 coarse cells per unit, cells within 0.6 of the re-entrant corner refined
        # once (2:1 hanging faces), degrees 1..4 in a 40/30/20/10 % mix: 108,149 elements
        return inputs.fichera_amr(20, radius=0.6)
    if name in ("obstacle-48", "obstacle-64"):
        n = int(name.split("-")[1])
        m = inputs.cavity(n, 2, name=f"obstacle_cavity_{n}x{n}x{n}_p2")
        inputs.sphere_obstacle(m, radius=0.2, eps=20.0 + 5.0j)
        return m
    if name == "obstacle":
        # unit cavity 32^3, p = 2, dielectric sphere eps = 20 + 5i of radius 0.2
        m = inputs.cavity(32, 2, name="obstacle_cavity_32x32x32_p2")
        inputs.sphere_obstacle(m, radius=0.2, eps=20.0 + 5.0j)
        return m
    raise ValueError(name)


def flops_factor_per_element(p):
    """Algorithmic FP64 flops of one element's factorisation and condensation.

    Cholesky of G (4 n_v^3 / 3), triangular solves with the m + 1 right-hand
    sides (4 n_v^2 (m+1)), the Gram product (4 n_v (m+1)^2) and the second
    condensation (4 n_u^3/3 + 4 n_u^2 (n_h+1) + 4 n_u (n_h+1)^2); complex
    multiply-add = 8 real flops, Hermitian halves counted once.
    """
    rt, r = p + 2, p + 1
    nv = 2 * 3 * rt * (rt + 1) ** 2
    nu = 6 * (p + 1) ** 3
    nh = 24 * r * r
    m1 = nu + nh + 1
    return (4 * nv ** 3 / 3 + 4 * nv ** 2 * m1 + 4 * nv * m1 ** 2
            + 4 * nu ** 3 / 3 + 4 * nu ** 2 * (nh + 1) + 4 * nu * (nh + 1) ** 2)


def tc_mma_flops_per_element(p, cplx):
    """FP16 tensor-core flops one element's split-arithmetic factorisation issues.

    The tile schedule of k_factor_tc: panels of 32 pivots (the first stage
    stops at n_v), then for the rows below a panel, 128-row blocks times
    NJ-column tiles up to the block's diagonal (NJ = 32 real, 16 complex);
    each tile takes the 28 digit pairs (a, b) with a + b <= 6 of the seven
    base-256 digits, each pair one 128 x NJ x 32 product (real) or four
    128 x 16 x 32 products (complex: real part over the stacked Re/Im
    columns, imaginary part as two cross products).  Equal to ncu's
    sm__ops_path_tensor_op_utchmma_src_fp16_dst_fp32 count on the 979-row
    p = 2 element.
    """
    rt, r = p + 2, p + 1
    nv = 2 * 3 * rt * (rt + 1) ** 2
    nu = 6 * (p + 1) ** 3
    nh = 24 * r * r
    N = nv + nu + nh + 1
    TB, TM = 32, 128
    NJ = 16 if cplx else 32
    per_tile = 28 * (8 * 2 * TM * NJ * 16 if cplx else 2 * 2 * TM * NJ * 16)
    k0, tot = 0, 0
    while k0 < nv + nu:
        k1 = k0 + min(TB, (nv if k0 < nv else nv + nu) - k0)
        R = N - k1
        for rho in range(0, R, TM):
            tot += (min(rho + TM, R) + NJ - 1) // NJ * per_tile
        k0 = k1
    return tot


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s, pw in zip(sm, power) if pw > 0.3 * max(power)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


def max_over_ranks(value, dist, device):
    """Max of a per-rank number over all ranks (all_reduce MAX); the number itself without a process group."""
    if not dist:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, n_elem, ms_step):
    """Whole-job elements/s: every rank solves its own replica of n_elem elements in ms_step (max over ranks)."""
    return world * n_elem / (ms_step / 1e3)


def _oracle_elements(task):
    """Worker of the CPU baseline: the oracle's element pass + recovery on a few elements (one BLAS thread)."""
    from oracle import element as oel
    from oracle import system as osys
    mesh, ids = task
    t0 = time.perf_counter()
    for e in ids:
        el = oel.element_matrices(mesh.vert[mesh.elem[e]], int(mesh.p[e]), mesh.omega, complex(mesh.eps[e]),
                                  complex(mesh.mu[e]), osys.element_faces(mesh, e))
        c = oel.condense(el)
        oel.recover(el, c, np.zeros(el.Bh.shape[1], complex))
    return time.perf_counter() - t0


class OraclePool:
    """Element-parallel CPU oracle: one process per host core (spawned, one BLAS thread each).

    The pool is started with the spawn method before any GPU work is done in
    the children, and every worker runs the oracle as it stands on its own
    share of the sampled elements.
    """

    def __init__(self, workers=None):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.workers = workers or max(1, min(os.cpu_count() or 1, 64))
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"
        self.pool = cf.ProcessPoolExecutor(max_workers=self.workers, mp_context=mp.get_context("spawn"))
        # start every worker and import the oracle there before anything is timed
        list(self.pool.map(_oracle_elements, [(None, []) for _ in range(self.workers)]))

    def rate(self, mesh, per_worker):
        """elements/s of the oracle over a sample of per_worker elements per process (wall clock)."""
        n_sample = per_worker * self.workers
        # the sample mixes boundary (port / impedance) and interior elements
        robin = np.where((mesh.face_bc == 2).any(axis=1))[0]
        inner = np.where(~(mesh.face_bc > 0).any(axis=1))[0]
        pick = list(robin[: max(1, n_sample // 4)]) + list(inner[: n_sample - max(1, n_sample // 4)])
        pick = (pick * (n_sample // max(1, len(pick)) + 1))[:n_sample]
        tasks = [(mesh, [int(e) for e in pick[k::self.workers]]) for k in range(self.workers)]
        t0 = time.perf_counter()
        list(self.pool.map(_oracle_elements, tasks))
        dt = time.perf_counter() - t0
        return len(pick) / dt, self.workers, dt, len(pick)

    def close(self):
        self.pool.shutdown()


def run_reference(args, rank):
    mesh = config_mesh(args.config)
    if rank != 0:
        return
    pool = OraclePool()
    vals = []
    for _ in range(args.warmup):
        pool.rate(mesh, args.ref_sample)
    for _ in range(args.steps):
        rate, cores, dt, n = pool.rate(mesh, args.ref_sample)
        vals.append((rate, dt))
    pool.close()
    rate = statistics.median(v[0] for v in vals)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(v[1] for v in vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": mesh.name, "elements": int(mesh.n_elem), "p": int(mesh.p[0]), "dp": 1},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} elements of {mesh.name} per step, {args.ref_sample} per process on "
                                       f"{cores} spawned processes with one BLAS thread each (element formation, "
                                       f"condensation, local recovery and eta_K); the global CG is not in the sample"},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="waveguide3d")
    ap.add_argument("--cg", default="auto", choices=["auto"] + sorted(CG_MODES),
                    help="auto: ir-bjacobi-ebe (element-by-element inner operator), ir-bjacobi when streaming")
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--inner-rtol", type=float, default=5e-2,
                    help="inner relative tolerance of iterative refinement (5e-2: the fewest total inner iterations "
                         "measured on the 32x16x64 guide, with either inner operator)")
    ap.add_argument("--max-iter", type=int, default=200000)
    ap.add_argument("--cpu-sample", type=int, default=2, help="oracle elements per host process (CPU baseline)")
    ap.add_argument("--ref-sample", type=int, default=1, help="oracle elements per host process per reference step")
    ap.add_argument("--no-fp64-arm", action="store_true",
                    help="skip the one-step FP64-throughout comparison arm after the timed steps")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=sorted(PRECISIONS))
    ap.add_argument("--chunk", type=int, default=0, help="elements per launch (0: library default)")
    ap.add_argument("--autotune", action="store_true", help="measure chunk sizes per degree before the warm-up")
    ap.add_argument("--bucketed", action="store_true",
                    help="order-bucketed element pass: waves of every order's chunks, persistent factorisation")
    ap.add_argument("--stream", action="store_true",
                    help="streaming element pass (no per-element condensation data; for the full-size configs)")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="after the timed steps, solve the same system with the plain FP64 CG and report it")
    ap.add_argument("--adjoint", action="store_true",
                    help="after the timed steps, time the adjoint gradient of the absorbed power (obstacle elements)")
    ap.add_argument("--adapt", type=int, default=0,
                    help="run the adaptive loop of Sec. 4.2 (fixed-fraction marking 0.30 / 0.05, 2:1 octree) on the "
                         "Fichera oven for this many adaptation steps instead of the timed steps")
    ap.add_argument("--adapt-p", type=int, default=2)
    ap.add_argument("--precision-report", action="store_true",
                    help="after the timed steps, solve again with FP64 quadrature and report the differences")
    args = ap.parse_args()
    streaming_cfg = args.stream or args.config in ("cavity3-32", "fichera-amr-1e5", "obstacle-48", "obstacle-64")
    if args.cg == "auto":  # the element-by-element operator needs every element's stored S_K
        args.cg = "ir-bjacobi" if streaming_cfg else "ir-bjacobi-ebe"

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    # the CPU baseline's process pool starts (spawn) before this process touches the GPU
    pool = OraclePool() if rank == 0 and not args.adapt else None

    import torch
    torch.cuda.set_device(local)
    if args.adapt:
        if pool:
            pool.close()
        return adaptive_run(args, rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2609_03155_b300 import dpg
    mesh = config_mesh(args.config)
    streaming = streaming_cfg
    d = dpg.DPG(mesh, precision=PRECISIONS[args.precision], chunk=args.chunk, adjoint=args.adjoint,
                streaming=streaming)
    mode = CG_MODES[args.cg]
    if not streaming:  # eta_K from the X = (L^-1 [B Bh l])^H the element pass keeps
        d.set_estimator_store(True)
    if args.bucketed:
        d.set_bucketed(True)
    tuned = d.autotune() if args.autotune else None
    stream = torch.cuda.current_stream()

    def step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        d.element_batch()
        ev[1].record(stream)
        d.assemble()
        ev[2].record(stream)
        x, rep = d.cg_solve(mode=mode, rtol=args.rtol, max_iter=args.max_iter, inner_rtol=args.inner_rtol,
                            raise_on_nonconvergence=False)
        ev[3].record(stream)
        u, eta, etag = d.estimate(x)
        ev[4].record(stream)
        return ev, rep, x, eta, etag

    try:
        for _ in range(args.warmup):
            step()
    except dpg.DPGError as err:
        if args.precision == "fp64":
            raise
        # reduced-precision quadrature can make G_K indefinite: report that and
        # the element-matrix differences instead of a throughput
        print(json.dumps({"metric": METRIC, "value": None, "unit": UNIT, "config": {"workload": mesh.name,
                          "quadrature": args.precision}, "error": str(err),
                          "precision_report": element_error_report(d, mesh)}), flush=True)
        return
    torch.cuda.synchronize()
    fp64, fp32 = dpg.probe_peaks()

    clk = ClockSampler(local)
    clk.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    d.timing_enable(True)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    phases = []
    for _ in range(args.steps):
        ev, rep, x, eta, etag = step()
        phases.append((ev, rep))
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    tim = d.timing_get()
    # SM-busy fraction of the timed pass's factorisation launches (per-element stamps)
    try:
        balance = {"mode": "order-bucketed persistent" if args.bucketed else "per-order chunks", **d.factor_balance()}
    except dpg.DPGError as err:
        balance = {"unavailable": str(err)}
    ms = max_over_ranks(t_start.elapsed_time(t_end), dist, "cuda")
    ms_step = ms / args.steps
    br = {"element_pass_s": [], "assemble_s": [], "cg_s": [], "estimate_s": []}
    for ev, rep in phases:
        br["element_pass_s"].append(ev[0].elapsed_time(ev[1]) / 1e3)
        br["assemble_s"].append(ev[1].elapsed_time(ev[2]) / 1e3)
        br["cg_s"].append(ev[2].elapsed_time(ev[3]) / 1e3)
        br["estimate_s"].append(ev[3].elapsed_time(ev[4]) / 1e3)
    br = {k: statistics.median(v) for k, v in br.items()}
    last_rep = phases[-1][1]

    # end to end through the public API: pinned host inputs in, solution out
    e2e = None
    if not args.no_e2e:
        corners = torch.from_numpy(np.ascontiguousarray(mesh.vert[mesh.elem].reshape(-1))).pin_memory()
        eps_h = torch.from_numpy(np.ascontiguousarray(mesh.eps)).pin_memory()
        mu_h = torch.from_numpy(np.ascontiguousarray(mesh.mu)).pin_memory()
        x_h = torch.empty(d.n, dtype=torch.complex128).pin_memory()
        eta_h = torch.empty(d.n_elem, dtype=torch.float64).pin_memory()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d.update_elements(corners, eps_h, mu_h)
        _, rep2, x2, eta2, _ = step()
        x_h.copy_(x2, non_blocking=True)
        eta_h.copy_(eta2, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
        e2e = {"value": job_throughput(world, mesh.n_elem, ems), "unit": UNIT,
               "h2d_bytes_per_step": int(corners.numel() * 8 + eps_h.numel() * 16 + mu_h.numel() * 16),
               "d2h_bytes_per_step": int(x_h.numel() * 16 + eta_h.numel() * 8)}

    if rank != 0:
        return
    p = int(mesh.p[0])
    pvals = sorted(set(int(q) for q in mesh.p))
    # element factorisation kernel (FP64 pipe): complex elements cost fpe(p)
    # flops, lossless (real-path) elements a quarter of that
    fpe = flops_factor_per_element(p)
    is_real = (mesh.eps.imag == 0) & (mesh.mu.imag == 0) & ~(mesh.face_bc == 2).any(axis=1)
    fpe_el = np.array([flops_factor_per_element(int(q)) for q in mesh.p]) * np.where(is_real, 0.25, 1.0)
    n_real = tim["factor_elements_real"]
    n_cplx = tim["factor_elements"] - n_real
    fac_avg_ms = tim["factor_ms"] / max(1, tim["factor_launches"])
    fac_flops = float(fpe_el.sum()) * tim["factor_elements"] / mesh.n_elem
    fac_achieved = fac_flops / max(1e-9, tim["factor_ms"] / 1e3) / 1e12
    common = {"flops_per_element_complex": fpe if len(pvals) == 1 else {str(q): flops_factor_per_element(q)
                                                                          for q in pvals},
              "flops_per_element_real": fpe / 4 if len(pvals) == 1 else "a quarter of the complex figure",
              "elements_real": n_real, "elements_complex": n_cplx, "launches": tim["factor_launches"],
              "avg_launch_ms": fac_avg_ms, "time_s": tim["factor_ms"] / 1e3}
    if d.factor_arith == 1:
        # trailing updates on the FP16 tensor cores through the exact digit
        # split: the ceiling is the tensor rate of the issued digit-pair MMAs
        # (FP16 runs at the bf16 rate); the FP64-equivalent rate is reported
        # beside it
        bf16_peak, bf16_src = 1800.0, "fallback 1.8 PFLOP/s bf16 (no MEASURED_PEAKS.json)"
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                bf16_peak = float(json.load(f)["bf16_tflops"])
                bf16_src = "MEASURED_PEAKS.json bf16_tflops (cuBLAS bf16 burst; FP16 MMAs run at the same rate)"
        except Exception:
            pass
        is_cplx = ~is_real
        tc_el = np.array([tc_mma_flops_per_element(int(q), bool(c)) for q, c in zip(mesh.p, is_cplx)], float)
        tc_flops = float(tc_el.sum()) * tim["factor_elements"] / mesh.n_elem
        tc_ach = tc_flops / max(1e-9, tim["factor_ms"] / 1e3) / 1e12
        roof_fac = {"bound": "tensor", "kernel": "k_factor_tc<double|double2> (blocked partial Cholesky + "
                    "condensation; trailing updates as FP16 digit-pair MMAs on tcgen05)",
                    "achieved": tc_ach, "peak": bf16_peak, "unit": "TFLOP/s", "frac": tc_ach / bf16_peak,
                    "peak_source": bf16_src, "traffic": None,
                    "mma_flops_rule": "28 digit pairs x 128-row tiles of the lower trailing triangle per panel",
                    "mma_flops_per_element_real": tc_mma_flops_per_element(p, False),
                    "mma_flops_per_element_complex": tc_mma_flops_per_element(p, True),
                    "fp64_equivalent_tflops": fac_achieved,
                    "fp64_equivalent_vs_dfma_peak": fac_achieved / (fp64 / 1e12),
                    "dfma_peak_tflops": fp64 / 1e12, **common}
    else:
        roof_fac = {"bound": "alu", "kernel": "k_factor<double|double2> (blocked partial Cholesky + condensation, "
                    "FP64 pipe)", "achieved": fac_achieved, "peak": fp64 / 1e12, "unit": "TFLOP/s",
                    "frac": fac_achieved / (fp64 / 1e12),
                    "peak_source": "FP64 FMA throughput measured live by dpg_probe_peaks (DFMA loop)",
                    "traffic": None, **common}
    # persistent CG kernel (HBM bound).  Algorithmic bytes per iteration
    # (the method's own traffic): the matrix values, 16 B per complex FP64
    # non-zero or 8 B per complex FP32 non-zero of the inner solves, plus six
    # vector passes; the column lists, the preconditioner's block inverses and
    # the further vector passes of this implementation are overhead, reported
    # apart.
    hbm_peak, hbm_src = 6400.0, "fallback 6.4 TB/s (no MEASURED_PEAKS.json)"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm_peak, hbm_src = float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured copy)"
    except Exception:
        pass
    bpi = d.cg_bytes_per_iteration(mode)
    vb = 8 if mode & 1 else 16
    # Hermitian half storage reads each off-diagonal block once: half the values
    mb = vb // 2 if mode & (16 | 128) else vb
    algo_bpi = mb * int(d.nnz) + 6 * vb * int(d.n)
    # DRAM traffic per iteration / implementation bytes of the FP32 inner CG
    # kernel, from the ncu capture of the 12x6x24 guide (dram__bytes_read.sum +
    # dram__bytes_write.sum over 279 iterations); the traffic per iteration
    # scales with the system, so a launch's traffic is this ratio times its bytes
    CG_TRAFFIC_RATIO_FP32 = 1.022
    # the same for the element-by-element operator (12x6x24 capture: 444 MB of
    # DRAM traffic per iteration against 450 MB of implementation bytes)
    CG_TRAFFIC_RATIO_EBE = 0.99
    cg_s = max(1e-9, tim["cg_kernel_ms"] / 1e3)
    cg_ach = algo_bpi * tim["cg_kernel_iterations"] / cg_s / 1e9
    spmv = ("element by element, FP32 upper-triangle tiles of S_K" if mode & 128 else
            "Hermitian half storage" if mode & 16 else "CSR rows")
    roof_cg = {"bound": "hbm", "kernel": "k_cg_persistent<%s> (one cooperative CG solve per launch; SpMV: %s)"
               % ("float2" if mode & 1 else "double2", spmv),
               "achieved": cg_ach, "peak": hbm_peak, "unit": "GB/s", "frac": cg_ach / hbm_peak,
               "traffic": ((CG_TRAFFIC_RATIO_EBE if mode & 128 else CG_TRAFFIC_RATIO_FP32) * bpi
                           * tim["cg_kernel_iterations"] / max(1, tim["cg_kernel_launches"])
                           if (mode & 1) and not (mode & 16) else None),
               "traffic_unit": "bytes per launch (ncu ratio %s x implementation bytes, from the 12x6x24 capture)"
                               % ("0.99" if mode & 128 else "1.022"),
               "peak_source": hbm_src, "bytes_per_iteration": algo_bpi,
               "bytes_rule": f"{mb} B x nnz + 6 x {vb} B x n (matrix values and six vector passes)",
               "overhead_bytes_per_iteration": bpi - algo_bpi,
               "overhead_rule": ("element tile padding and the overlap of element matrices, the trace-slot "
                                 "gathers, products and lists, block-Jacobi inverses and the other vector passes"
                                 if mode & 128 else
                                 "per-entity column lists, block-Jacobi inverses and the other vector passes"),
               "achieved_with_overhead": bpi * tim["cg_kernel_iterations"] / cg_s / 1e9,
               "iterations": tim["cg_kernel_iterations"], "launches": tim["cg_kernel_launches"],
               "avg_launch_ms": tim["cg_kernel_ms"] / max(1, tim["cg_kernel_launches"]),
               "time_s": tim["cg_kernel_ms"] / 1e3}
    if roof_cg["time_s"] >= roof_fac["time_s"]:
        roof, roof2 = roof_cg, roof_fac
    else:
        roof, roof2 = roof_fac, roof_cg
    cg_iters = last_rep["iterations"]
    # the FP64-throughout arm (the paper's solver: plain FP64 CG from x0 = 0),
    # one whole step end to end, and the complex-path element rate
    fp64_arm = None if args.no_fp64_arm else fp64_step(d, mesh, x, args)
    complex_rate = complex_path_rate(mesh, args) if args.config == "waveguide3d" else None
    rate, cores, dt, nsamp = pool.rate(mesh, args.cpu_sample)
    pool.close()
    line = {
        "metric": METRIC, "value": job_throughput(world, mesh.n_elem, ms_step), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("f64" if not (mode & 1) else "f64+f32(IR inner)")
        + ("" if args.precision == "fp64" else f"+{args.precision}(quadrature)"),
        "data": "synthetic",
        "config": {"workload": mesh.name, "elements": int(mesh.n_elem),
                   "p": p if len(pvals) == 1 else {str(q): int((mesh.p == q).sum()) for q in pvals}, "dp": 1,
                   "quadrature": args.precision,
                   "chunks": {str(g[0]): g[2] for g in d.group_info()} if d.h else None,
                   "autotuned": tuned is not None, "streaming": streaming, "bucketed": args.bucketed,
                   "estimator": ("L^-1 r_K from the stored L^-1 [B Bh l]" if not streaming
                                 else "L^-1 r_K by a second (recondensing) element pass"),
                   "trace_unknowns": int(d.n), "nnz": int(d.nnz), "cg": args.cg, "cg_rtol": args.rtol,
                   "cg_inner_rtol": args.inner_rtol,
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (per-element stores and CSR are tens of GB)"},
        "breakdown": {**br, "element_pass_elements_per_s": mesh.n_elem / br["element_pass_s"],
                      "cg_time_to_rtol_s": br["cg_s"], "cg_iterations": cg_iters, "cg_outer": last_rep["outer"],
                      "cg_rel_residual": last_rep["rel_residual"], "cg_converged": last_rep["converged"],
                      "cg_ms_per_iteration": 1e3 * br["cg_s"] / max(1, cg_iters)},
        "fp64_arm": fp64_arm,
        "complex_path_element_pass": complex_rate,
        "factor_load_balance": balance,
        "roofline": roof,
        "roofline_secondary": roof2,
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{nsamp} elements of {mesh.name} ({dt:.1f} s wall), {args.cpu_sample} per process "
                                   f"on {cores} spawned processes with one BLAS thread each: element formation, "
                                   f"condensation, recovery and eta_K; CG not in the sample"},
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": int(tim["kernel_launches"]),
        "peaks_measured": {"fp64_tflops": fp64 / 1e12, "fp32_tflops": fp32 / 1e12},
    }
    if args.compare_fp64:
        line["fp64_comparison"] = fp64_comparison(d, x, args)
    if args.adjoint:
        line["adjoint"] = adjoint_timing(d, mesh, x, args)
    if args.precision_report and args.precision != "fp64":
        line["precision_report"] = precision_report(d, mesh, x, eta, mode, args)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def adaptive_run(args, rank):
    """The adaptive loop of Sec. 4.2 on the Fichera oven: estimate, mark (fixed fractions 0.30 / 0.05), refine /
    coarsen a 2:1 octree, set up again; one JSON line with the per-step sizes, estimates and device times."""
    import torch
    from paper_2609_03155_b300 import dpg, inputs
    tree = inputs.fichera_octree(p=args.adapt_p)
    mode = CG_MODES[args.cg]
    stream = torch.cuda.current_stream()
    steps = []
    for step in range(args.adapt + 1):
        mesh, leaves = tree.mesh()
        t0 = time.perf_counter()
        d = dpg.DPG(mesh)
        setup_s = time.perf_counter() - t0
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        d.element_batch()
        ev[1].record(stream)
        d.assemble()
        ev[2].record(stream)
        x, rep = d.cg_solve(mode=mode, rtol=args.rtol, max_iter=args.max_iter, inner_rtol=args.inner_rtol,
                            raise_on_nonconvergence=False)
        ev[3].record(stream)
        _, eta, etag = d.estimate(x, want_u=False)
        ev[4].record(stream)
        torch.cuda.synchronize()
        marks = d.mark_fraction(eta, 0.30, 0.05, power=1)
        levels = sorted({c[0] for c in leaves})
        steps.append({"step": step, "elements": int(mesh.n_elem), "trace_unknowns": int(d.n), "nnz": int(d.nnz),
                      "levels": [int(levels[0]), int(levels[-1])], "global_estimate": etag,
                      "refine": int((marks > 0).sum()), "coarsen": int((marks < 0).sum()),
                      "setup_s": setup_s, "element_pass_s": ev[0].elapsed_time(ev[1]) / 1e3,
                      "assemble_s": ev[1].elapsed_time(ev[2]) / 1e3, "cg_s": ev[2].elapsed_time(ev[3]) / 1e3,
                      "cg_iterations": rep["iterations"], "cg_rel_residual": rep["rel_residual"],
                      "estimate_s": ev[3].elapsed_time(ev[4]) / 1e3})
        d.destroy()
        if step < args.adapt:
            tree.adapt(leaves, marks)
    if rank == 0:
        tot_el = sum(s["elements"] for s in steps)
        dev_s = sum(s["element_pass_s"] + s["assemble_s"] + s["cg_s"] + s["estimate_s"] for s in steps)
        print(json.dumps({"metric": METRIC, "value": tot_el / dev_s, "unit": UNIT, "n_gpus": 1,
                          "higher_is_better": True, "dtype": "f64+f32(IR inner)", "data": "synthetic",
                          "config": {"workload": f"fichera_oven_adaptive_p{args.adapt_p}", "adaptation_steps": args.adapt,
                                     "marking": "fixed fraction 0.30 refine / 0.05 coarsen of sum eta_K",
                                     "cg": args.cg, "cg_rtol": args.rtol},
                          "adaptive": steps}), flush=True)


def fp64_step(d, mesh, x_mixed, args):
    """One whole step in FP64 throughout: FP64 quadrature and factorisation, the paper's solver (plain FP64 CG,
    x0 = 0, no preconditioner).

    Timed end to end like e2e (pinned host inputs in, solution and eta out),
    with CUDA events around each phase; value = elements / device time of the
    step without the copies.  Also the relative L2 difference of its trace
    solution from the timed (mixed-precision) step's.
    """
    import torch
    corners = torch.from_numpy(np.ascontiguousarray(mesh.vert[mesh.elem].reshape(-1))).pin_memory()
    eps_h = torch.from_numpy(np.ascontiguousarray(mesh.eps)).pin_memory()
    mu_h = torch.from_numpy(np.ascontiguousarray(mesh.mu)).pin_memory()
    x_h = torch.empty(d.n, dtype=torch.complex128).pin_memory()
    eta_h = torch.empty(d.n_elem, dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream()
    # FP64 throughout: the factorisation's trailing updates on the FP64 pipe too
    d.set_factor_arith(0)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
    ev[0].record(stream)
    d.update_elements(corners, eps_h, mu_h)
    ev[1].record(stream)
    d.element_batch()
    ev[2].record(stream)
    d.assemble()
    ev[3].record(stream)
    x64, rep = d.cg_solve(mode=CG_MODES["fp64"], rtol=args.rtol, max_iter=args.max_iter,
                          raise_on_nonconvergence=False)
    ev[4].record(stream)
    _, eta64, _ = d.estimate(x64)
    ev[5].record(stream)
    x_h.copy_(x64, non_blocking=True)
    eta_h.copy_(eta64, non_blocking=True)
    ev[6].record(stream)
    torch.cuda.synchronize()
    d.set_factor_arith(1)
    dev_ms = ev[1].elapsed_time(ev[5])
    e2e_ms = ev[0].elapsed_time(ev[6])
    diff = float(torch.linalg.vector_norm(x_mixed - x64) / torch.linalg.vector_norm(x64))
    return {"cg": "fp64 (unpreconditioned, x0 = 0: the paper's solver)", "quadrature": "fp64",
            "factorisation": "fp64 (trailing updates on the FP64 pipe)",
            "value": mesh.n_elem / (dev_ms / 1e3), "unit": UNIT, "ms_per_step": dev_ms,
            "element_pass_s": ev[1].elapsed_time(ev[2]) / 1e3, "assemble_s": ev[2].elapsed_time(ev[3]) / 1e3,
            "cg_time_to_rtol_s": ev[3].elapsed_time(ev[4]) / 1e3, "estimate_s": ev[4].elapsed_time(ev[5]) / 1e3,
            "cg_iterations": rep["iterations"], "cg_rel_residual": rep["rel_residual"],
            "cg_converged": rep["converged"],
            "cg_ms_per_iteration": ev[3].elapsed_time(ev[4]) / max(1, rep["iterations"]),
            "e2e": {"value": mesh.n_elem / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": int(corners.numel() * 8 + eps_h.numel() * 16 + mu_h.numel() * 16),
                    "d2h_bytes_per_step": int(x_h.numel() * 16 + eta_h.numel() * 8)},
            "solution_rel_l2_difference_vs_timed_step": diff,
            "note": "one step after the timed region; both arms stop at the same FP64 relative residual"}


def complex_path_rate(mesh, args):
    """Element pass with every element on the complex path (real path off), on a 4-cell slab of the same guide.

    The slab's elements have the shape, size, materials and frequency of the
    full guide's, so its per-element rate is the full guide's complex-path rate.
    """
    import torch
    from paper_2609_03155_b300 import dpg, inputs
    p = int(mesh.p[0])
    nx, ny, nz = mesh.grid if getattr(mesh, "grid", None) else (32, 16, 64)
    slab = inputs.waveguide(0.08636, 0.04318, 0.300 * 4 / nz, nx, ny, 4, 2.45e9, p, name="waveguide3d_slab")
    d = dpg.DPG(slab)
    d.set_real_path(False)
    d.element_batch()
    torch.cuda.synchronize()
    d.timing_enable(True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    d.element_batch()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    tim = d.timing_get()
    d.destroy()
    fpe = flops_factor_per_element(p)
    return {"elements": int(slab.n_elem), "workload": f"{nx}x{ny}x4 slab of the same guide, real path off",
            "elements_per_s": slab.n_elem / (ms / 1e3), "element_pass_s": ms / 1e3,
            "factor_fp64_equivalent_tflops": fpe * tim["factor_elements"] / max(1e-9, tim["factor_ms"] / 1e3) / 1e12}


def fp64_comparison(d, x, args):
    """The paper's solver (plain FP64 CG, x0 = 0) on the same assembled system, against the timed solution."""
    import torch
    x64, rep = d.cg_solve(mode=CG_MODES["fp64"], rtol=args.rtol, max_iter=args.max_iter,
                          raise_on_nonconvergence=False)
    diff = float(torch.linalg.vector_norm(x - x64) / torch.linalg.vector_norm(x64))
    return {"cg": "fp64 (unpreconditioned, the paper's solver)", "time_s": rep["ms"] / 1e3,
            "iterations": rep["iterations"], "rel_residual": rep["rel_residual"], "converged": rep["converged"],
            "solution_rel_l2_difference": diff}


def adjoint_timing(d, mesh, x, args):
    """P and dP/deps of the elements with Im eps > 0 (the obstacle): one adjoint CG and one gradient pass."""
    import torch
    mask = torch.tensor((mesh.eps.imag > 0).astype(np.uint8), device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P, dre, dim = d.grad_eps(x, mask, cg_mode=CG_MODES[args.cg], rtol=args.rtol, max_iter=args.max_iter)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"P": P, "time_s": dt, "obstacle_elements": int(mask.sum().item()),
            "grad_abs_max": float(torch.maximum(dre.abs().max(), dim.abs().max()).item()),
            "cg": args.cg, "cg_rtol": args.rtol}


def element_error_report(d, mesh):
    """G, B, S of sampled elements in the handle's precision against FP64 quadrature."""
    from paper_2609_03155_b300 import dpg
    ids = np.linspace(0, mesh.n_elem - 1, 8).astype(np.int32)
    ids = ids[mesh.p[ids] == mesh.p[ids[0]]]
    red = d.element_dump(ids)
    d.destroy()
    ref = dpg.DPG(mesh)
    full = ref.element_dump(ids)
    ref.destroy()
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    # smallest eigenvalue of each sampled G_K relative to its largest (FP64 and reduced)
    lam = lambda G: float(min(np.linalg.eigvalsh(g)[0] / np.linalg.eigvalsh(g)[-1] for g in G))
    return {"elements_sampled": int(len(ids)), "G_rel_frobenius": rel(red["G"], full["G"]),
            "B_rel_frobenius": rel(red["B"], full["B"]), "min_eig_ratio_G_fp64": lam(full["G"]),
            "min_eig_ratio_G_reduced": lam(red["G"]),
            "reference": "same elements, FP64 quadrature"}


def precision_report(d, mesh, x, eta, mode, args):
    """Differences of the reduced-precision run against FP64 quadrature on the same mesh."""
    import torch
    from paper_2609_03155_b300 import dpg
    ids = np.linspace(0, mesh.n_elem - 1, 8).astype(np.int32)
    ids = ids[mesh.p[ids] == mesh.p[ids[0]]]
    red = d.element_dump(ids)
    x_red = x.cpu().numpy()
    eta_red = eta.cpu().numpy()
    d.destroy()
    ref = dpg.DPG(mesh)
    full = ref.element_dump(ids)
    ref.element_batch()
    ref.assemble()
    t0 = time.perf_counter()
    x64, _ = ref.cg_solve(mode=mode, rtol=args.rtol, max_iter=args.max_iter, inner_rtol=args.inner_rtol)
    _, eta64, _ = ref.estimate(x64)
    x64 = x64.cpu().numpy()
    eta64 = eta64.cpu().numpy()
    ref.destroy()
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    return {"elements_sampled": int(len(ids)),
            "G_rel_frobenius": rel(red["G"], full["G"]), "B_rel_frobenius": rel(red["B"], full["B"]),
            "S_rel_frobenius": rel(red["S"], full["S"]),
            "trace_solution_rel_l2": rel(x_red, x64), "eta_rel_l2": rel(eta_red, eta64),
            "reference": "same mesh, FP64 quadrature, same CG mode and tolerance"}


if __name__ == "__main__":
    main()
