#!/usr/bin/env python
"""Benchmark of the FMM-BEM hot path on GB300.

Workload (one step): the two FMM passes of one direct-formulation mat-vec
on a 4,000,000-point bumpy-sphere surface point set -- a Laplace apply and a
Yukawa (kappa = 0.125) apply, each with single-layer (monopole) and
double-layer (dipole, per-point unit normals) sources, expansion order
p = 6, ncrit = 128, FP32 arithmetic (PB_MIXED).  Metric: FMM apply
points/s = targets evaluated per apply per second (2 applies per step).

Lines printed (one JSON line on rank 0):
  --impl ours       (default) the CUDA path through the C-ABI
  --impl reference  the FP64 direct-sum oracle on the host cores, on a
                    bounded target sample per step (this run's reference arm)
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_POINTS = 4_000_000
P_ORDER = 6
NCRIT = 128
KAPPA = 0.125
METRIC = "FMM apply points/s (4M-point surface, Laplace+Yukawa SL+DL, p=6)"
UNIT = "points/s"
# dram__bytes_read.sum + dram__bytes_write.sum of one leaf launch
# (k_leaf_pair_x2) on this workload (4M points, p = 6, ncrit = 128), from one
# ncu capture of the current kernel (505.6 + 27.2 MB, direct W/X lists on);
# None once the kernel changes
LEAF_TRAFFIC_BYTES = 532.8e6
# Arithmetic of one source-target pair in the paired (Laplace + Yukawa)
# evaluation, FMA = 2 FLOPs, MUFU counted apart: SL+DL of both kernels
# 30 FLOPs + 2 MUFU (rsqrt, ex2); monopole-only pairs of equivalent
# densities (M2P, L2P) 16 FLOPs + 2 MUFU.
FLOPS_PAIR = {"pair_sd": 30, "pair_m": 16}
MUFU_PAIR = 2


def max_over_ranks(ms, dist):
    """The slowest rank's step time (the job's time); plain value at N = 1.
    Reduced on the GPU under NCCL, on the host under gloo."""
    if dist is None:
        return ms
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def list_work(ex, ne, direct_w, direct_x):
    """Pair counts of the leaf kernel when the adaptive-list pairs are taken
    directly where that is less work (PB_OPT_LIST_DIRECT): W-list boxes of at
    most ne // 2 sources, and the X list of a leaf of at most ne targets.
    Returns (direct W pairs, direct X pairs, M2P targets left, P2L sources
    left)."""
    nchild = ex["nchild"]
    ns = (ex["src_end"] - ex["src_begin"]).astype(np.int64)
    nt = (ex["tgt_end"] - ex["tgt_begin"]).astype(np.int64)
    if nt.sum() == 0:                        # targets = sources
        nt = ns
    woff, wids = ex["W"]
    xoff, xids = ex["X"]
    rw = np.repeat(np.arange(len(nchild)), np.diff(woff))
    rx = np.repeat(np.arange(len(nchild)), np.diff(xoff))
    dw = (ns[wids] <= ne // 2) if direct_w else np.zeros(len(wids), bool)
    dx = ((nchild[rx] == 0) & (nt[rx] <= ne)) if direct_x else np.zeros(len(xids), bool)
    return (int((nt[rw] * ns[wids])[dw].sum()), int((nt[rx] * ns[xids])[dx].sum()),
            int(nt[rw][~dw].sum()), int(ns[xids][~dx].sum()))


def job_throughput(world, n_points, ms):
    """Whole-job points/s: every rank (replica) evaluates both kernels at its
    own n_points targets per step of ms milliseconds (weak scaling)."""
    return world * 2 * n_points / (ms * 1e-3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_POINTS)
    ap.add_argument("--p", type=int, default=P_ORDER)
    ap.add_argument("--ncrit", type=int, default=NCRIT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--virus", action="store_true", help="virus-scale shell solve only (10M triangles, 1.6M atoms)")
    ap.add_argument("--virus-face", type=int, default=645, help="cube-sphere subdivision (12 n^2 triangles per wall)")
    ap.add_argument("--virus-atoms", type=int, default=1_600_000)
    ap.add_argument("--virus-fp64", action="store_true",
                    help="with --virus: also solve the shell with the all-FP64 GPU path and compare dG")
    ap.add_argument("--sweep", action="store_true", help="p x ncrit grid of the 4M-point apply")
    ap.add_argument("--profile", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--tc-kernel", choices=["pair", "single"], default=None,
                    help="tensor-core box-operator kernel: CTA pairs (cta_group::2) or one CTA per operator part "
                         "(default: the library's choice)")
    ap.add_argument("--binding", type=int, default=0, metavar="N",
                    help="batched binding energies of N synthetic complexes (compact receptor 500-5,000 atoms, "
                         "ligand 20-300 atoms; 3N meshes) in one pb_solve_batch")
    ap.add_argument("--binding-form", choices=["exterior", "direct"], default="direct",
                    help="formulation of --binding: exterior derivative (P1, Eq. lu) or direct (P0)")
    ap.add_argument("--kirkwood", action="store_true",
                    help="off-centre-charge sphere refinement study (512 ... 131,072 elements)")
    ap.add_argument("--leaf-nt", type=int, default=0, choices=[0, 2, 4],
                    help="targets per thread of the leaf kernel (PB_OPT_LEAF_NT; 0: the library's default)")
    ap.add_argument("--list-direct", type=int, default=1, choices=[0, 1, 2, 3],
                    help="PB_OPT_LIST_DIRECT: 0 every W/X pair through the equivalent surfaces, 1 small W boxes "
                         "and small leaves' X lists directly, 2 X lists only, 3 W boxes only")
    ap.add_argument("--leaf-scalar", action="store_true",
                    help="scalar FP32 leaf kernel instead of the packed f32x2 one (PB_OPT_LEAF_PACKED 0)")
    return ap.parse_args()


def inputs(n):
    import synthetic
    x, nrm = synthetic.bumpy_sphere_points(n, seed=0)
    q = synthetic.uniform_densities(n, seed=1)
    d = synthetic.uniform_densities(n, seed=2)
    return x, nrm, q, d


def select_tc_kernel(pb, choice):
    """Apply --tc-kernel and return the kernel in use ("pair" or "single")."""
    if choice is not None:
        pb._test_tc_pair(1 if choice == "pair" else 0)
        return choice
    mode = pb._test_tc_pair(0)
    pb._test_tc_pair(mode)
    return "pair" if mode else "single"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_sample(x, nrm, q, d, ntgt, seed=5):
    """FP64 direct sums (the oracle as it stands) for a target sample; returns seconds."""
    import synthetic
    from oracle.kernels import LAPLACE, YUKAWA, direct_sum
    idx = synthetic.random_subsample(len(x), ntgt, seed=seed)
    t0 = time.perf_counter()
    direct_sum(LAPLACE, 0.0, x, q=q, dip=d, src_n=nrm, tgt=x[idx])
    direct_sum(YUKAWA, KAPPA, x, q=q, dip=d, src_n=nrm, tgt=x[idx])
    return time.perf_counter() - t0


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([s.strip() for s in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.3)
            self.proc.terminate()
            self.proc.wait()
            self.thread.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if len(s) > 2 and s[1].replace('.', '', 1).isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) > 2 and s[2].replace('.', '', 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, nm in enumerate(names):
                if len(s) > 5 + k and s[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def workload_config(args, world):
    """The workload both arms report (the GPU arm adds the tree's sizes)."""
    return {"workload": f"fmm_apply_pair {args.n} bumpy-sphere points (amp 0.05), Laplace+Yukawa "
                        f"(kappa {KAPPA}) SL+DL in one traversal, p={args.p}, ncrit={args.ncrit}, tree cached",
            "global_batch": args.n * world, "seq_len": None,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "flushed between steps (256 MB write)"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    x, nrm, q, d = inputs(args.n)
    ntgt = 400
    for _ in range(args.warmup):
        oracle_sample(x, nrm, q, d, ntgt)
    ts = [oracle_sample(x, nrm, q, d, ntgt, seed=100 + k) for k in range(args.steps)]
    t = float(np.mean(ts))
    value = 2 * ntgt / t
    cores = host_cores()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"FP64 direct sums (the oracle as it stands) at {ntgt} sampled targets "
                                       f"x {args.n} sources x 2 kernels per step",
                             "cpu": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_virus(args):
    """Virus-scale shell: 1.6M atoms, ~10M triangles, one mixed-precision
    solve (p = 4, 3-point rule, GMRES tol 1e-4 as the paper's Zika run)."""
    import torch
    import paper_2103_01048_gb300 as pb
    import synthetic
    def note(msg):
        print(f"[virus {time.perf_counter() - t_start:8.1f} s] {msg}", file=sys.stderr, flush=True)

    t_start = t0 = time.perf_counter()
    V, T, xyz, radii, q = synthetic.virus_shell(n_atoms=args.virus_atoms, n_face=args.virus_face)
    t_gen = time.perf_counter() - t0
    note(f"generated {len(T)} triangles, {len(q)} atoms")
    ctx = pb.pb_create(0, None)
    free0, total = torch.cuda.mem_get_info()
    pb.pb_profile(ctx, True)
    t0 = time.perf_counter()
    mesh = pb.pb_mesh_setup(ctx, V, T, 3, 4, 128)
    nt = len(T)
    x = np.zeros(2 * nt)
    y = np.zeros(2 * nt)
    note("mesh set up")
    pb.pb_mesh_matvec(ctx, mesh, x, y, 4.0, 80.0, 0.125)        # assembles S, builds the operators
    t_setup = time.perf_counter() - t0
    setup_prof = pb.pb_profile_read(ctx)
    pb.pb_profile(ctx, False)
    note(f"singular entries + operators + first mat-vec: {t_setup:.1f} s")
    t0 = time.perf_counter()
    res, st = pb.pb_solve(ctx, mesh, xyz, q, 4.0, 80.0, 0.125, 1e-4, 300)
    t_solve = time.perf_counter() - t0
    note(f"solve: {t_solve:.1f} s")
    t0 = time.perf_counter()
    e = pb.pb_solvation_energy(ctx, res)
    t_energy = time.perf_counter() - t0
    it, rr, _ = pb.pb_result_get(res)
    free1, _ = torch.cuda.mem_get_info()
    line = {"metric": "PB solve s per mesh (virus-scale shell)", "value": t_solve + t_energy, "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f32 FMM / f64 GMRES", "data": "synthetic",
            "config": {"workload": f"virus-scale shell: {len(q)} atoms, {nt} triangles ({3 * nt} quadrature "
                                   f"points), two cube-sphere walls r=230/270 A, p=4, ncrit=128, tol 1e-4",
                       "singular_rule": "FP64 5-level" if nt <= 262144 else "FP32 4-level"},
            "setup_profile_ms": {k: round(v[0], 1) for k, v in setup_prof.items()
                                 if k != "launches" and v[0] > 0},
            "status": int(st), "iterations": it, "residual": rr, "dG_kcal_mol": e,
            "setup_s": t_setup, "solve_s": t_solve, "energy_s": t_energy, "generate_s": t_gen,
            "ms_per_gmres_iteration": 1e3 * t_solve / max(it, 1),
            "device_gb_in_use_after": (total - free1) / 1e9, "device_gb_in_use_before": (total - free0) / 1e9,
            "paper_context": "Zika (~10M elements, direct): GMRES 9470.9 s, 105 iterations, 109.7 GB, "
                             "dual 20-core Xeon Gold 6148"}
    if args.virus_fp64:
        # the same mesh, charges and tolerance on the all-FP64 path (FP64
        # FMM, operators and GMRES): dG agreement of the mixed path at scale
        t0 = time.perf_counter()
        res64, st64 = pb.pb_solve(ctx, mesh, xyz, q, 4.0, 80.0, 0.125, 1e-4, 300, precision=pb.PB_FP64)
        t64 = time.perf_counter() - t0
        e64 = pb.pb_solvation_energy(ctx, res64)
        it64, rr64, _ = pb.pb_result_get(res64)
        line["fp64"] = {"status": int(st64), "iterations": it64, "residual": rr64, "dG_kcal_mol": e64,
                        "solve_s": t64}
        line["mixed_vs_fp64_rel_dG"] = abs(e - e64) / abs(e64)
        line["speedup_mixed_over_fp64"] = t64 / t_solve
        note(f"FP64 solve: {t64:.1f} s, rel dG {line['mixed_vs_fp64_rel_dG']:.2e}")
        pb.pb_result_destroy(res64)
    print(json.dumps(line), flush=True)
    pb.pb_result_destroy(res)
    pb.pb_mesh_destroy(mesh)
    pb.pb_destroy(ctx)


def _gen_complex(spec):
    import synthetic as syn
    n_rec, n_lig, seed = spec
    return spec, syn.binding_complex(n_rec, n_lig, seed=seed, dense=True)


def run_binding(args):
    """Batched binding energies (Eq. bind) at scale: N seeded synthetic
    complexes (compact receptor of 500-5,000 atoms, ligand of 20-300 atoms,
    atom centres 4.5 A apart at the closest), the complex, receptor and
    ligand surfaces of each (3N meshes) solved together by one pb_solve_batch
    (mixed precision, p = 6, tol 1e-5, eps 4/80, kappa 0.125).  Reports the
    host mesh generation, the library set-up (mesh set-up, singular entries,
    operators shared between trees of equal box sizes), the batched solve
    and the binding energies; one JSON line."""
    import multiprocessing as mp
    rng = np.random.default_rng(2021)
    specs = [(int(rng.integers(500, 5001)), int(rng.integers(20, 301)), 5000 + c) for c in range(args.binding)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(max(1, min(len(specs), host_cores()))) as pool:
        gen = pool.map(_gen_complex, specs)
    t_gen = time.perf_counter() - t0
    import torch
    import paper_2103_01048_gb300 as pb
    C = 332.0637
    ctx = pb.pb_create(0, None)
    # singular entries with the FP32 4-level rule for every mesh (the FP64
    # 5-level rule, the default below 262,144 triangles, runs at the FP64
    # rate); its effect on dG is measured on one ligand below
    pb.pb_set_option(ctx, pb.PB_OPT_SINGULAR, 2)
    ext = args.binding_form == "exterior"
    form = pb.PB_FORM_EXTERIOR if ext else pb.PB_FORM_DIRECT
    basis = pb.PB_P1 if ext else pb.PB_P0
    # GMRES(200) with up to 800 iterations in all: 201 Krylov vectors per
    # system; keep the complexes whose estimated footprint fits: the basis
    # (201 x 2 n doubles) plus ~7 KB per triangle of singular entries, trees
    # and workspaces (an overestimate: 139 GB measured for 18.7M triangles
    # with 251 vectors)
    max_iter, restart = 800, 200
    pb.pb_set_option(ctx, pb.PB_OPT_RESTART, restart)
    free, _ = torch.cuda.mem_get_info()
    per_tri = 16 * (restart + 1) * (0.5 if ext else 1.0) + 7000
    keep, used = [], 0.0
    for spec, cx in gen:
        need = per_tri * sum(len(cx["surf"][k][1]) for k in ("cplx", "rec", "lig"))
        if used + need > 0.75 * free:
            break
        keep.append((spec, cx))
        used += need
    dropped = len(gen) - len(keep)
    gen = keep
    meshes, atoms_l, q_l, coul = [], [], [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for spec, cx in gen:
        for k in ("cplx", "rec", "lig"):
            V, T = cx["surf"][k]
            meshes.append(pb.pb_mesh_setup(ctx, V, T.astype(np.int32), 3, 6, 64, basis=basis))
            atoms_l.append(cx[k][0]); q_l.append(cx[k][2])
        xr, xl = cx["rec"][0], cx["lig"][0]
        r = np.linalg.norm(xr[:, None, :] - xl[None, :, :], axis=2)
        coul.append(C * (cx["rec"][2][:, None] * cx["lig"][2][None, :] / (4.0 * r)).sum())
    torch.cuda.synchronize()
    t_mesh = time.perf_counter() - t0
    ntri = [pb.pb_mesh_info(m)[0] for m in meshes]
    # set-up: one preconditioned mat-vec per mesh builds its singular
    # entries, tree lists and (shared) operator sets
    t0 = time.perf_counter()
    for m in meshes:
        nu = pb.pb_mesh_unknowns(m)
        xv = torch.zeros(2 * nu, dtype=torch.float64, device="cuda")
        yv = torch.empty_like(xv)
        pb.pb_mesh_matvec(ctx, m, xv, yv, 4.0, 80.0, 0.125, precond=True, formulation=form)
    torch.cuda.synchronize()
    t_first = time.perf_counter() - t0
    t0 = time.perf_counter()
    res_l, sts, rc = pb.pb_solve_batch(ctx, meshes, atoms_l, q_l, 4.0, 80.0, 0.125, 1e-5, max_iter,
                                       formulation=form)
    t_batch = time.perf_counter() - t0
    eb = [pb.pb_solvation_energy(ctx, r_) for r_ in res_l]
    got = [pb.pb_result_get(r_)[:2] for r_ in res_l]
    iters = [int(g_[0]) for g_ in got]
    unconv = [{"triangles": ntri[i], "iterations": iters[i], "residual": float(got[i][1])}
              for i in range(len(res_l)) if sts[i] != pb.PB_OK]
    for r_ in res_l:
        pb.pb_result_destroy(r_)
    n = len(gen)
    dgb = [eb[3 * c] - eb[3 * c + 1] - eb[3 * c + 2] - coul[c] for c in range(n)]
    # the FP32 singular rule against the FP64 one on the smallest mesh
    k = int(np.argmin(ntri))
    pb.pb_set_option(ctx, pb.PB_OPT_SINGULAR, 1)
    r64, _ = pb.pb_solve(ctx, meshes[k], atoms_l[k], q_l[k], 4.0, 80.0, 0.125, 1e-5, max_iter, formulation=form)
    e64 = pb.pb_solvation_energy(ctx, r64)
    pb.pb_result_destroy(r64)
    sing = {"mesh_triangles": ntri[k], "dG_fp32_rule": eb[k], "dG_fp64_rule": e64,
            "rel_diff": abs(eb[k] - e64) / abs(e64)}
    line = {"metric": "batched binding energies, ms per mesh", "value": t_batch * 1e3 / len(meshes),
            "unit": "ms/mesh", "higher_is_better": False, "n_gpus": 1, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"{n} synthetic complexes (compact receptor 500-5,000 atoms, ligand 20-300) x (complex, "
                                   f"receptor, ligand) = {len(meshes)} meshes, {min(ntri)}-{max(ntri)} triangles "
                                   f"({sum(ntri)} in all), "
                                   + ("exterior derivative formulation (Eq. lu), P1" if ext else
                                      "direct formulation, P0")
                                   + ", p = 6, mixed, GMRES(200) to tol 1e-5, eps 4/80, kappa 0.125, FP32 "
                                     "singular rule, one pb_solve_batch"},
            "singular_rule_check": sing, "complexes_generated": n + dropped,
            "complexes_dropped_for_memory": dropped, "device_free_gb_at_start": free / 1e9,
               "host_generation_s": t_gen, "mesh_setup_s": t_mesh,
               "setup_s_singular_lists_operators": t_first, "batched_solve_s": t_batch, "max_iter": max_iter,
               "gmres_restart": restart, "unconverged": unconv,
               "status_ok": int(sum(1 for s_ in sts if s_ == pb.PB_OK)), "rc": int(rc),
               "iterations": {"min": min(iters), "median": float(np.median(iters)), "max": max(iters)},
               "dG_bind_kcal_mol": {"min": float(min(dgb)), "median": float(np.median(dgb)), "max": float(max(dgb))},
               "dG_bind_first3": dgb[:3]}
    print(json.dumps(line), flush=True)
    for m in meshes:
        pb.pb_mesh_destroy(m)
    pb.pb_destroy(ctx)


def run_kirkwood(args):
    """Sphere of radius 4 A with a unit charge at (1, 1, 1), eps 4 / 80,
    kappa 0.125: octahedral meshes of 512 ... 131,072 elements, 6-point rule,
    p = 10, GMRES tol 1e-7 (the paper's refinement study); error against
    Kirkwood's series and the observed order from the middle three meshes."""
    import torch
    import paper_2103_01048_gb300 as pb
    import synthetic
    # the paper's analytic (Kirkwood) value and parameters, a cited golden file
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                                       "kirkwood_sphere.json")))
    g = {"radius": gold["radius"], "q": gold["q"], "pos": gold["position"], "eps_in": gold["eps_in"],
         "eps_out": gold["eps_out"], "kappa": gold["kappa"]}
    E_k = gold["energy_kcal_mol"]
    ctx = pb.pb_create(0, None)
    rows = []
    for lev in (3, 4, 5, 6, 7):
        V, F = synthetic.octasphere(lev, g["radius"])
        t0 = time.perf_counter()
        mesh = pb.pb_mesh_setup(ctx, V, F.astype(np.int32), 6, 10, 128)
        res, st = pb.pb_solve(ctx, mesh, np.array([g["pos"]]), np.array([g["q"]]), g["eps_in"], g["eps_out"],
                              g["kappa"], 1e-7, 500)
        pb.pb_result_destroy(res)
        t_setup = time.perf_counter() - t0          # includes operators and singular entries
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res, st = pb.pb_solve(ctx, mesh, np.array([g["pos"]]), np.array([g["q"]]), g["eps_in"], g["eps_out"],
                              g["kappa"], 1e-7, 500)
        E = pb.pb_solvation_energy(ctx, res)
        t_solve = (time.perf_counter() - t0) * 1e3
        it, rr, _ = pb.pb_result_get(res)
        pb.pb_result_destroy(res)
        pb.pb_mesh_destroy(mesh)
        rows.append({"elements": len(F), "dG_kcal_mol": E, "rel_error": abs(E - E_k) / abs(E_k), "iterations": it,
                     "status": int(st), "solve_ms": t_solve, "first_solve_s": t_setup})
        print(f"[kirkwood] {len(F)} elements: dG {E:.6f}, rel err {rows[-1]['rel_error']:.3e}, {it} it, "
              f"{t_solve:.1f} ms", file=sys.stderr, flush=True)
    n = np.array([r["elements"] for r in rows], dtype=np.float64)
    e = np.array([r["rel_error"] for r in rows])
    order = float(-np.polyfit(np.log(n[1:4]), np.log(e[1:4]), 1)[0])
    line = {"metric": "Kirkwood sphere relative dG error (vs the paper's analytic value), finest mesh",
            "value": rows[-1]["rel_error"],
            "unit": "relative", "higher_is_better": False, "n_gpus": 1, "dtype": "f32 FMM / f64 GMRES",
            "data": "synthetic",
            "config": {"workload": "sphere r = 4 A, +1 e at (1,1,1), eps 4/80, kappa 0.125, octahedral meshes "
                                   "512-131,072 elements, 6-point rule, p = 10, tol 1e-7"},
            "analytic_dG_kcal_mol": E_k,
            "observed_order_middle_three": order, "paper_observed_order": 1.001, "meshes": rows}
    print(json.dumps(line), flush=True)
    pb.pb_destroy(ctx)


def run_sweep(args):
    """The expansion orders and leaf sizes of the 4M-point FMM workload:
    paired apply (Laplace + Yukawa SL+DL) at p = 4, 6, 8, 10 and ncrit =
    64, 128, 256, ms per apply (median of 5 after 2 warm-ups, L2 flushed),
    tree build and operator set-up time; one JSON line."""
    import torch
    import paper_2103_01048_gb300 as pb
    tc_kernel = select_tc_kernel(pb, args.tc_kernel)
    x, nrm, q, d = inputs(args.n)
    stream = torch.cuda.Stream()
    ctx = pb.pb_create(0, stream)
    X, Nr, Q, D = (torch.from_numpy(a).cuda() for a in (x, nrm, q, d))
    out_l = torch.empty(args.n, device="cuda")
    out_y = torch.empty(args.n, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda")
    rows = []
    for ncrit in (64, 128, 256):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tree = pb.fmm_tree_build(ctx, X, ncrit)
        t_tree = (time.perf_counter() - t0) * 1e3
        info = pb.fmm_tree_info(tree)
        for p in (4, 6, 8, 10):
            t0 = time.perf_counter()
            pb.fmm_apply_pair(ctx, tree, KAPPA, p, out_l, out_y, q_lap=Q, q_yuk=Q, dip=D, src_n=Nr)
            pb.pb_sync(ctx)
            t_first = time.perf_counter() - t0
            pb.fmm_apply_pair(ctx, tree, KAPPA, p, out_l, out_y, q_lap=Q, q_yuk=Q, dip=D, src_n=Nr)
            ts = []
            for k in range(5):
                with torch.cuda.stream(stream):
                    flush.fill_(float(k))
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    pb.fmm_apply_pair(ctx, tree, KAPPA, p, out_l, out_y, q_lap=Q, q_yuk=Q, dip=D, src_n=Nr)
                    b.record(stream)
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            pb.pb_sync(ctx)
            ms = float(np.median(ts))
            rows.append({"p": p, "ncrit": ncrit, "ms_per_paired_apply": ms, "points_per_s": 2 * args.n / (ms * 1e-3),
                         "first_apply_s_incl_operators": t_first, "tree_build_ms": t_tree,
                         "boxes": info.n_box, "levels": info.n_levels, "v_pairs": info.n_v})
            print(f"[sweep] ncrit {ncrit} p {p}: {ms:.2f} ms, first apply {t_first:.1f} s", file=sys.stderr,
                  flush=True)
        pb.fmm_tree_destroy(tree)
    print(json.dumps({"metric": "FMM apply points/s over the expansion orders and leaf sizes",
                      "unit": "points/s", "n_gpus": 1, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": f"fmm_apply_pair {args.n} bumpy-sphere points, Laplace+Yukawa "
                                             f"(kappa {KAPPA}) SL+DL", "l2": "flushed between applies",
                                 "tc_kernel": tc_kernel},
                      "rows": rows}), flush=True)
    pb.pb_destroy(ctx)


def main():
    args = parse()
    if args.sweep:
        return run_sweep(args)
    if args.virus:
        return run_virus(args)
    if args.kirkwood:
        return run_kirkwood(args)
    if args.binding:
        return run_binding(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import paper_2103_01048_gb300 as pb
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    tc_kernel = select_tc_kernel(pb, args.tc_kernel)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    # the CPU baseline runs before any GPU work on rank 0 (bounded sample)
    x, nrm, q, d = inputs(args.n)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ntgt = 2000
        t = oracle_sample(x, nrm, q, d, ntgt)
        cpu = {"value": 2 * ntgt / t, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
               "sample": f"{ntgt} targets x {args.n} sources, FP64 direct sum, Laplace+Yukawa SL+DL "
                         f"({t:.1f} s)", "cpu": cpu_model()}

    # measured arithmetic peaks of this GPU (the roofline denominators), with
    # the SM clock sampled while they run
    with Clocks(local) as clk_pk:
        peaks = pb.measure_peaks(local)
    peaks["clocks"] = clk_pk.summary()
    peaks["how"] = ("pbfmm_measure_peaks: dependent-chain FP32/FP64 FMA and MUFU rsqrt/ex2 loops on every SM, "
                    "tcgen05.mma M128 N256 (kind::tf32 and kind::f16 BF16) with operands resident in shared "
                    "memory; CUDA events")

    stream = torch.cuda.Stream()
    ctx = pb.pb_create(local, stream)
    pb.pb_set_option(ctx, pb.PB_OPT_LEAF_NT, args.leaf_nt)
    pb.pb_set_option(ctx, pb.PB_OPT_LEAF_PACKED, 0 if args.leaf_scalar else 1)
    pb.pb_set_option(ctx, pb.PB_OPT_LIST_DIRECT, args.list_direct)
    X = torch.from_numpy(x).cuda()
    Nr = torch.from_numpy(nrm).cuda()
    Q = torch.from_numpy(q).cuda()
    D = torch.from_numpy(d).cuda()
    # tree build (a1-a2: keys, radix sort, boxes, lists), reported apart from
    # the apply as in the paper's assembly / solve split: the median of 3
    # builds after one warm-up build
    t_builds = []
    for k in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tree = pb.fmm_tree_build(ctx, X, args.ncrit)
        torch.cuda.synchronize()
        if k > 0:
            t_builds.append((time.perf_counter() - t0) * 1e3)
        if k < 3:
            pb.fmm_tree_destroy(tree)
    tree_build_ms = float(np.median(t_builds))
    info = pb.fmm_tree_info(tree)
    out_l = torch.empty(args.n, device="cuda")
    out_y = torch.empty(args.n, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda")

    def step():
        pb.fmm_apply_pair(ctx, tree, KAPPA, args.p, out_l, out_y, q_lap=Q, q_yuk=Q, dip=D, src_n=Nr)

    def step_two_applies():
        pb.fmm_apply(ctx, tree, pb.FMM_LAPLACE, 0.0, args.p, out_l, q=Q, dip=D, src_n=Nr)
        pb.fmm_apply(ctx, tree, pb.FMM_YUKAWA, KAPPA, args.p, out_y, q=Q, dip=D, src_n=Nr)

    # warm-up (also builds and caches the operators)
    for _ in range(max(args.warmup, 3)):
        step()
    pb.pb_sync(ctx)
    torch.cuda.synchronize()

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    pb.pb_profile(ctx, True)
    if args.profile:
        torch.cuda.cudart().cudaProfilerStart()
    with Clocks(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))            # L2 flush between timed steps (untimed)
                ev[k][0].record(stream)
                step()
                ev[k][1].record(stream)
        torch.cuda.synchronize()
    if args.profile:
        torch.cuda.cudart().cudaProfilerStop()
    prof = pb.pb_profile_read(ctx)
    pb.pb_profile(ctx, False)
    if dist:
        dist.barrier()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / args.steps, dist)
    value = job_throughput(world, args.n, ms)

    # the same work as two single-kernel applies (for comparison; untimed by the metric)
    for _ in range(2):
        step_two_applies()
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
    for k in range(3):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
            ev2[k][0].record(stream)
            step_two_applies()
            ev2[k][1].record(stream)
    torch.cuda.synchronize()
    ms_two = sum(a.elapsed_time(b) for a, b in ev2) / 3

    # e2e through the C-ABI with pinned host buffers (H2D of inputs, D2H of results inside)
    hq = torch.from_numpy(q).pin_memory()
    hd = torch.from_numpy(d).pin_memory()
    hn = torch.from_numpy(nrm).pin_memory()
    ho_l = torch.empty(args.n).pin_memory()
    ho_y = torch.empty(args.n).pin_memory()

    def step_host():
        pb.fmm_apply_pair(ctx, tree, KAPPA, args.p, ho_l, ho_y, q_lap=hq, q_yuk=hq, dip=hd, src_n=hn)

    step_host()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_host()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, dist)
    h2d = q.nbytes + d.nbytes + nrm.nbytes              # q_lap and q_yuk are one host array, staged once
    d2h = 2 * 4 * args.n

    # roofline of the dominant phase (per-launch averages from the library's event timers)
    phases = {k: v for k, v in prof.items() if k != "launches" and v[1] > 0}
    dom = max(phases, key=lambda k: phases[k][0])
    # leaf phase per step: one launch, or with the stream overlap option the
    # near-field launch (second stream) plus the far-field launch, each timed
    # by CUDA events on its own stream
    leaf_ms = phases["leaf"][0] / args.steps
    p = args.p
    ne = 6 * (p - 1) ** 2 + 2
    on = not args.leaf_scalar and args.list_direct != 0 and ne <= 1024
    w_dir, x_dir, m2p_left, p2l_left = list_work(pb.fmm_tree_export(ctx, tree), ne, on and args.list_direct != 2,
                                                 on and args.list_direct != 3)
    near = info.p2p_pairs + w_dir + x_dir
    far = (m2p_left + info.l2p_targets) * ne
    leaf_flops = near * FLOPS_PAIR["pair_sd"] + far * FLOPS_PAIR["pair_m"]
    leaf_mufu = (near + far) * MUFU_PAIR
    fma_peak = peaks["fp32_fma_tflops"] * 1e12                        # FLOP/s, measured
    # one rsqrt and one ex2 per pair, on the same MUFU unit: the harmonic mean
    mufu_peak = 2.0 / (1.0 / peaks["mufu_rsqrt_tops"] + 1.0 / peaks["mufu_ex2_tops"]) * 1e12
    t_roof = max(leaf_flops / fma_peak, leaf_mufu / mufu_peak)       # s per launch at the ALU roof
    achieved = leaf_flops / (leaf_ms * 1e-3) / 1e12
    peak = leaf_flops / t_roof / 1e12
    split = phases["leaf"][1] > args.steps        # near/far launches on two streams (PB_OPT_OVERLAP)
    leaf_kernel = "k_leaf_pair" if args.leaf_scalar else "k_leaf_pair_x2 (packed f32x2)"
    roof = {"kernel": (f"{leaf_kernel} near (P2P, second stream) + far (M2P/L2P) launches per step" if split
                       else f"{leaf_kernel}: P2P+M2P+L2P, Laplace+Yukawa"),
            "bound": "alu", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": LEAF_TRAFFIC_BYTES if (LEAF_TRAFFIC_BYTES and args.n == N_POINTS and args.p == P_ORDER
                                              and args.ncrit == NCRIT) else None,
            "traffic_note": "DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum); "
                            "the launch streams each target leaf's U-list sources (~0.56 GB, L2-filtered)",
            "peak_note": "ALU roof of this launch's instruction mix from the peaks measured in this run: "
                         "FLOPs / max(FLOPs / FP32 FMA peak, MUFU ops / MUFU peak); the MUFU peak is the "
                         "harmonic mean of the measured rsqrt and ex2 rates (one of each per pair)",
            "fma_frac": leaf_flops / (leaf_ms * 1e-3) / fma_peak,
            "mufu_frac": leaf_mufu / (leaf_ms * 1e-3) / mufu_peak,
            "dominant_phase": dom}
    launches = prof["launches"]
    # M2L on the tensor cores: algorithmic FLOPs 2 n_e^2 per V-list pair and
    # kernel (the un-split product) against the measured TF32 rate
    m2l_ms = phases["m2l"][0] / args.steps if "m2l" in phases else None
    roof_m2l = None
    if m2l_ms:
        npad = (ne + 31) // 32 * 32
        m2l_flops = 2 * 2.0 * ne * ne * info.n_v
        roof_m2l = {"kernel": "k_m2l_tc (tcgen05 kind::tf32, Laplace+Yukawa in one launch)", "bound": "tensor",
                    "achieved": m2l_flops / (m2l_ms * 1e-3) / 1e12, "peak": peaks["tf32_tc_tflops"],
                    "unit": "TFLOP/s", "frac": m2l_flops / (m2l_ms * 1e-3) / 1e12 / peaks["tf32_tc_tflops"],
                    "issued_frac": 3 * 2 * 2.0 * npad * npad * info.n_v / (m2l_ms * 1e-3) / 1e12
                    / peaks["tf32_tc_tflops"],
                    "frac_of_fp32_accurate_roof": m2l_flops / (m2l_ms * 1e-3) / 1e12
                    / (peaks["tf32_tc_tflops"] / 3.0),
                    "note": "achieved = 2 n_e^2 x V-list pairs x 2 kernels / M2L phase time; issued_frac counts "
                            "the 3 TF32 products (hi*hi, hi*lo, lo*hi) at the padded size n_pad actually issued; "
                            "frac_of_fp32_accurate_roof divides by TF32 / 3, the rate of a contraction that keeps "
                            "FP32 accuracy with three TF32 products"}

    clocks = clk.summary()

    # PB solve ms per mesh, mixed vs all-FP64 GPU path, at equal expansion
    # order: the Born ion (5,120-triangle icosphere of radius 2 A, +1e at the
    # centre, P0, 3-point rule, GMRES tol 1e-6) at p = 4, 5, 6, each energy
    # against the dense-LU oracle's (a golden value written by
    # tests/golden/make_born_ion.py); setup excluded (as the paper's
    # assembly/solve split).  Headline: the lowest p at which both arms are
    # within 1e-4 of the oracle.  Then the 2,000-atom synthetic protein
    # (~80,000 triangles, tol 1e-5) at p = 6, mixed vs FP64.
    solve = None
    if rank == 0 and not args.no_solve:
        import synthetic as syn
        gold = json.load(open(os.path.join(ROOT, "tests", "golden", "born_ion_5120.json")))
        e_or = gold["energy_kcal_mol"]
        V, F = syn.icosphere(4, 2.0)
        atoms, qa = np.zeros((1, 3)), np.array([1.0])
        solve = {"workload": "Born ion r=2 A, 5120 triangles, 3-pt rule, P0, tol 1e-6, eps 4/80, kappa 0.125",
                 "oracle_dG_kcal_mol": e_or, "by_p": {}}

        def timed_solve(mesh, a_, q_, prec, tol, reps, formulation=pb.PB_FORM_DIRECT):
            res, st = pb.pb_solve(ctx, mesh, a_, q_, 4.0, 80.0, 0.125, tol, 500, precision=prec,
                                  formulation=formulation)
            pb.pb_result_destroy(res)                     # warm: operators, singular entries, graph
            ts = []
            for _ in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                res, st = pb.pb_solve(ctx, mesh, a_, q_, 4.0, 80.0, 0.125, tol, 500, precision=prec,
                                      formulation=formulation)
                e = pb.pb_solvation_energy(ctx, res)
                ts.append((time.perf_counter() - t0) * 1e3)
                it, rr, _ = pb.pb_result_get(res)
                pb.pb_result_destroy(res)
            return {"ms_per_mesh": float(np.median(ts)), "iterations": it, "dG_kcal_mol": e, "status": int(st)}

        for p_s in (4, 5, 6):
            mesh = pb.pb_mesh_setup(ctx, V, F.astype(np.int32), 3, p_s, 128)
            row = {}
            for name, prec in (("mixed", pb.PB_MIXED), ("fp64", pb.PB_FP64)):
                row[name] = timed_solve(mesh, atoms, qa, prec, 1e-6, 3)
                row[name]["rel_dG_vs_oracle"] = abs(row[name]["dG_kcal_mol"] - e_or) / abs(e_or)
            row["speedup_mixed_over_fp64"] = row["fp64"]["ms_per_mesh"] / row["mixed"]["ms_per_mesh"]
            solve["by_p"][str(p_s)] = row
            pb.pb_mesh_destroy(mesh)
        ok = [int(k) for k, r in solve["by_p"].items()
              if r["mixed"]["rel_dG_vs_oracle"] <= 1e-4 and r["fp64"]["rel_dG_vs_oracle"] <= 1e-4]
        hp = str(min(ok)) if ok else "6"
        solve["headline_p"] = int(hp)
        solve["mixed"] = dict(solve["by_p"][hp]["mixed"], p=int(hp))
        solve["fp64"] = dict(solve["by_p"][hp]["fp64"], p=int(hp))
        solve["speedup_mixed_over_fp64"] = solve["by_p"][hp]["speedup_mixed_over_fp64"]
        solve["mixed_vs_fp64_rel_dG"] = abs(solve["mixed"]["dG_kcal_mol"] - solve["fp64"]["dG_kcal_mol"]) / abs(
            solve["fp64"]["dG_kcal_mol"])
        # the synthetic protein (2,000 atoms, ~80,000 triangles)
        Vp, Tp, xyz_p, _, q_p, _ = syn.synthetic_protein()
        mesh = pb.pb_mesh_setup(ctx, Vp, Tp.astype(np.int32), 3, 6, 128)
        prot = {"workload": f"synthetic protein: 2000 atoms, {len(Tp)} triangles, 3-pt rule, P0, p=6, ncrit=128, "
                            f"tol 1e-5, eps 4/80, kappa 0.125"}
        for name, prec in (("mixed", pb.PB_MIXED), ("fp64", pb.PB_FP64)):
            prot[name] = timed_solve(mesh, xyz_p, q_p, prec, 1e-5, 1)
        pb.pb_mesh_destroy(mesh)
        prot["mixed_vs_fp64_rel_dG"] = abs(prot["mixed"]["dG_kcal_mol"] - prot["fp64"]["dG_kcal_mol"]) / abs(
            prot["fp64"]["dG_kcal_mol"])
        prot["speedup_mixed_over_fp64"] = prot["fp64"]["ms_per_mesh"] / prot["mixed"]["ms_per_mesh"]
        solve["protein"] = prot
        # the exterior derivative formulation (Eq. lu, P1, lumped-mass
        # preconditioner) on the same two surfaces: iterations and ms per
        # mesh beside the direct formulation's
        # Born's closed form for a unit charge at the centre of a sphere of
        # radius a = 2 A: (q^2 / 2a) (1 / (eps_out (1 + kappa a)) - 1 / eps_in) C
        born = 0.5 * (1.0 / (80.0 * (1 + 0.125 * 2.0)) - 1.0 / 4.0) / 2.0 * 332.0637
        deriv = {"workload": "exterior derivative formulation (Eq. lu), P1, lumped-mass preconditioner, "
                             "same meshes, p and tolerances as the direct rows",
                 "born_closed_form_kcal_mol": born}
        mesh = pb.pb_mesh_setup(ctx, V, F.astype(np.int32), 3, int(hp), 128, basis=pb.PB_P1)
        for name, prec in (("mixed", pb.PB_MIXED), ("fp64", pb.PB_FP64)):
            r = timed_solve(mesh, atoms, qa, prec, 1e-6, 3, formulation=pb.PB_FORM_EXTERIOR)
            r["rel_dG_vs_born"] = abs(r["dG_kcal_mol"] - born) / abs(born)
            deriv["born_" + name] = r
        pb.pb_mesh_destroy(mesh)
        deriv["born_direct_rel_dG_vs_born"] = abs(solve["mixed"]["dG_kcal_mol"] - born) / abs(born)
        mesh = pb.pb_mesh_setup(ctx, Vp, Tp.astype(np.int32), 3, 6, 128, basis=pb.PB_P1)
        deriv["protein_mixed"] = timed_solve(mesh, xyz_p, q_p, pb.PB_MIXED, 1e-5, 1, formulation=pb.PB_FORM_EXTERIOR)
        pb.pb_mesh_destroy(mesh)
        deriv["protein_rel_dG_exterior_P1_vs_direct_P0"] = abs(
            deriv["protein_mixed"]["dG_kcal_mol"] - prot["mixed"]["dG_kcal_mol"]) / abs(prot["mixed"]["dG_kcal_mol"])
        solve["derivative"] = deriv

    # batched binding energies: complexes -> (complex, receptor, ligand)
    # meshes solved together by pb_solve_batch vs one at a time
    batch = None
    if rank == 0 and not args.no_solve:
        import synthetic as syn
        C = 332.0637
        meshes, atoms_l, q_l, tags = [], [], [], []
        ncx = 3
        for c in range(ncx):
            cx = syn.binding_complex(150 + 60 * c, 15 + 5 * c, seed=10 + c)
            for k in ("cplx", "rec", "lig"):
                V, T = cx["surf"][k]
                meshes.append(pb.pb_mesh_setup(ctx, V, T.astype(np.int32), 3, 6, 64))
                atoms_l.append(cx[k][0]); q_l.append(cx[k][2]); tags.append((c, k))
            xr, xl = cx["rec"][0], cx["lig"][0]
            r = np.linalg.norm(xr[:, None, :] - xl[None, :, :], axis=2)
            tags.append(("coul", c, C * (cx["rec"][2][:, None] * cx["lig"][2][None, :] / (4.0 * r)).sum()))
        ntri = [pb.pb_mesh_info(m)[0] for m in meshes]
        # warm (operators, singular entries)
        res_l, _, _ = pb.pb_solve_batch(ctx, meshes, atoms_l, q_l, 4.0, 80.0, 0.125, 1e-5, 500)
        for r_ in res_l:
            pb.pb_result_destroy(r_)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res_l, sts, rc = pb.pb_solve_batch(ctx, meshes, atoms_l, q_l, 4.0, 80.0, 0.125, 1e-5, 500)
        t_batch = (time.perf_counter() - t0) * 1e3
        eb = [pb.pb_solvation_energy(ctx, r_) for r_ in res_l]
        for r_ in res_l:
            pb.pb_result_destroy(r_)
        t0 = time.perf_counter()
        es = []
        for m, a_, q_ in zip(meshes, atoms_l, q_l):
            r_, _ = pb.pb_solve(ctx, m, a_, q_, 4.0, 80.0, 0.125, 1e-5, 500)
            es.append(pb.pb_solvation_energy(ctx, r_))
            pb.pb_result_destroy(r_)
        t_seq = (time.perf_counter() - t0) * 1e3
        coul = {t[1]: t[2] for t in tags if t[0] == "coul"}
        # Eq. bind: dG_bind = dG_complex - dG_receptor - dG_ligand - dG_coul
        dgb = [eb[3 * c] - eb[3 * c + 1] - eb[3 * c + 2] - coul[c] for c in range(ncx)]
        batch = {"workload": f"{ncx} synthetic complexes x (complex, receptor, ligand) = {len(meshes)} meshes, "
                             f"{min(ntri)}-{max(ntri)} triangles, mixed, tol 1e-5",
                 "batched_ms_per_mesh": t_batch / len(meshes), "sequential_ms_per_mesh": t_seq / len(meshes),
                 "speedup": t_seq / t_batch,
                 "max_rel_dG_batched_vs_sequential": float(max(abs(a - b) / abs(b) for a, b in zip(eb, es))),
                 "dG_bind_kcal_mol": dgb,
                 "dG_coul_eps_in_kcal_mol": [coul[c] for c in range(ncx)]}
        for m in meshes:
            pb.pb_mesh_destroy(m)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(workload_config(args, world), tc_kernel=tc_kernel),
                "tree": {"boxes": info.n_box, "leaves": info.n_leaf, "levels": info.n_levels,
                         "v_pairs": info.n_v, "p2p_pairs": info.p2p_pairs, "m2p_targets": info.m2p_targets,
                         "p2l_sources": info.p2l_sources, "l2p_targets": info.l2p_targets,
                         "build_ms": tree_build_ms,
                         "direct_w_pairs": w_dir, "direct_x_pairs": x_dir, "m2p_targets_far": m2p_left,
                         "p2l_sources_far": p2l_left,
                         "direct_note": "pairs of W-list boxes of at most n_e/2 sources and of the X lists of leaves "
                                        "of at most n_e targets are summed directly in the leaf kernel "
                                        "(PB_OPT_LIST_DIRECT); m2p_targets_far / p2l_sources_far are the rest",
                         "build_note": "fmm_tree_build wall time with a device synchronisation, median of 3 "
                                       "after one warm-up build; not part of the timed step (tree cached)"},
                "paired_step_points_per_s": value / 2,
                "metric_note": "value counts both kernels' targets (2 x n per paired step); one direct-"
                               "formulation mat-vec's FMM work is one paired step: paired_step_points_per_s",
                "roofline": roof, "roofline_m2l": roof_m2l, "peaks": peaks, "cpu_baseline": cpu,
                "e2e": {"value": job_throughput(world, args.n, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": int(launches), "clocks": clocks, "pb_solve": solve, "pb_solve_batch": batch,
                "phases_ms_per_step": {k: v[0] / args.steps for k, v in phases.items()},
                "phases_note": "CUDA-event time per phase on the stream it runs on",
                "two_applies_ms_per_step": ms_two}
        print(json.dumps(line), flush=True)
    pb.fmm_tree_destroy(tree)
    pb.pb_destroy(ctx)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
