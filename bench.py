"""Benchmark of the randomized-multiplier GENP solve (Pan, Qian, Yan, arXiv:1406.5802) on GB300.

One step = the whole hot path on one system: draw the Gaussian multiplier G (Def. 4.1), form
M = A G (Fact 4.1), factor M by blocked GENP (Sec. 3), solve and recover X = G Y, and refine to
normwise backward error <= 1e-13 (Sec. 7.1), all through the librmge C ABI.

Workload: n = 4096, A = U diag(sigma) V^T with U, V Haar-orthogonal and sigma log-spaced 1 .. 1e-6,
B 4096 x 16 i.i.d. N(0,1), FP64 (the paper's orthogonal-factor test matrices, Sec. 7.1, at this size).
Inputs are larger than L2 (A, G and M are 134 MB each).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  N > 1 runs as torchrun replicas: each rank solves its own system,
no collective on the data path (weak scaling).  --impl reference times the CPU FP64 oracle on the
host cores instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s & TFLOP/s of A·G GENP solve at backward err ≤1e-13, mixed vs FP64"
N_SYS, K_RHS, SIGMA_MIN = 4096, 16, 1e-6
SEED = 0x5EED0000 + 2
BE_TOL, MAX_ITERS = 1e-13, 10
# FP64 on GB300 runs on the DFMA pipe: 2 DFMA per clock per SM (measured 1.195 TFLOP/s with an
# FMA-chain microbenchmark); the nominal peak at the 2070 MHz maximum SM clock is
# 152 SMs x 2 DFMA x 2 flop x 2.070 GHz = 1.2586 TFLOP/s.
FP64_ALU_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# DRAM bytes (read + write) of one A G launch at n = 4096, from an ncu capture of this kernel
# (dram__bytes_read.sum + dram__bytes_write.sum); reset to None whenever the kernel changes.
AG_TRAFFIC_BYTES = 3.730475e9 + 0.134292e9
# The same for the emulated-FP64 A G kernel of the mixed form (oz_gemm_kernel) at n = 4096.
OZ_AG_TRAFFIC_BYTES = 2.203738e9 + 0.185977e9


def flops_per_solve(n, k, sweeps):
    """Algorithmic flops: A G (2n^3 - n^2), GENP (2n^3/3 - n^2/2 - n/6), L, U solves + X = G Y
    (4n^2 k), and per refinement sweep the residual (2n^2 k) plus the correction (4n^2 k)."""
    return (2 * n**3 - n**2) + (2 * n**3 / 3 - n**2 / 2 - n / 6) + 4 * n**2 * k + sweeps * 6 * n**2 * k


def sample_clocks(stop, out):
    cmd = ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]]
    while not stop.is_set():
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=5)
            if r.returncode == 0 and r.stdout.strip():
                out.append([t.strip() for t in r.stdout.strip().splitlines()[0].split(",")])
        except Exception:
            pass
        stop.wait(0.2)


def clocks_summary(samples):
    if not samples:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    sm = [float(s[0]) for s in samples if s[0].replace(".", "").isdigit()]
    mx = [float(s[1]) for s in samples if s[1].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for s in samples for i in range(4) if len(s) > 3 + i and s[3 + i] == "Active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(samples)}


def cpu_oracle_solve(A, B, G, threads):
    from oracle import oracle as orc
    orc.set_threads(threads)
    t0 = time.perf_counter()
    out = orc.rmge_solve(orc.GAUSSIAN, A, G, B, max_iters=MAX_ITERS, be_tol=BE_TOL)
    dt = time.perf_counter() - t0
    return dt, out


def host_inputs():
    from paper_1406_5802_gb300 import workloads as W
    import numpy as np
    A, B = W.orthogonal_factor_system(N_SYS, K_RHS, SIGMA_MIN, seed=SEED)
    return np.ascontiguousarray(A), np.ascontiguousarray(B)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as orc
    cores = os.cpu_count() or 1
    A, B = host_inputs()
    G = orc.gaussian(N_SYS * N_SYS, SEED, 1).reshape(N_SYS, N_SYS)
    times, sweeps = [], 0
    for i in range(args.warmup + args.steps):
        dt, out = cpu_oracle_solve(A, B, G, cores)
        if i >= args.warmup:
            times.append(dt)
            sweeps = out["iters"]
    t = sum(times) / len(times)
    value = 1.0 / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "randomized GENP solve, n=4096, 16 RHS, FP64, Gaussian multiplier",
                       "n": N_SYS, "nrhs": K_RHS, "sigma": "log-spaced 1..1e-6", "precision": "f64"},
            "tflops": flops_per_solve(N_SYS, K_RHS, sweeps) * value / 1e12,
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full n=4096 oracle solves (plain C, OpenMP rows)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def extra_workloads(W, rmge, peaks, which=("precision", "batch", "grad", "lowrank")):
    """The other measured workloads (one JSON object each, added to the main line): the n = 16384
    precision comparison (the FP64 form against the tensor-core forms with FP64 refinement: emulated FP64
    products (f64x), three-pass and one-pass BF16/FP16 splits), the batch of 4096 uneven systems in one
    persistent graph-captured launch, and the differentiable batch of 64 systems."""
    import numpy as np
    import torch

    out = {}

    def ev():
        return torch.cuda.Event(enable_timing=True)

    # -- precision: n = 16384, sigma 1 .. 1e-4, 8 RHS -------------------------------------------------
    try:
        if "precision" not in which:
            raise LookupError("not selected")
        n, k = 16384, 8
        A, B = W.orthogonal_factor_system_torch(n, k, 1e-4, seed=W.SEED_BASE + 3, device="cuda")
        res = {"workload": "n=16384, 8 RHS, A = U diag(sigma) V^T, sigma log-spaced 1..1e-4, Gaussian G"}
        for prec in ("f64", "f64x", "bf16x3", "f16x3", "bf16"):
            ws = rmge.workspace(n, k, "gaussian", prec)
            G = rmge.empty_multiplier("gaussian", n, prec)
            M = torch.empty(n, n, dtype=rmge.factor_dtype(prec), device="cuda")
            X = torch.empty(n, k, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0, t1, a0, a1 = ev(), ev(), ev(), ev()
            t0.record()
            rmge.make_multiplier("gaussian", n, W.SEED_BASE + 3, 1, prec, G=G)
            a0.record()
            rmge.apply_multiplier("gaussian", A, G, prec, M=M, ws=ws)
            a1.record()
            info, growth = rmge.factor(M, prec, ws=ws)
            rmge.solve("gaussian", M, G, B, prec, X=X, ws=ws)
            berr, iters = rmge.refine("gaussian", A, M, G, B, X, prec, 10, 1e-13, ws=ws)
            t1.record()
            torch.cuda.synchronize()
            it = int(iters.item())
            ms, ams = t0.elapsed_time(t1), a0.elapsed_time(a1)
            terms = {"f64": 1, "f64x": 36, "bf16x3": 3, "f16x3": 3, "bf16": 1}[prec]
            entry = {"ms_per_solve": ms, "solves_per_s": 1e3 / ms, "berr_final": float(berr[it].item()),
                     "sweeps": it, "reached_1e-13": bool(berr[it].item() <= 1e-13), "growth": float(growth.item()),
                     "info": int(info.item()), "apply_ms": ams,
                     "tflops_algorithmic": flops_per_solve(n, k, it) / (ms / 1e3) / 1e12}
            if prec != "f64":
                tc_tflops = terms * 2 * n**3 / (ams / 1e3) / 1e12
                entry["apply_tensor_tflops"] = tc_tflops
                entry["apply_tensor_frac_of_bf16_peak"] = tc_tflops / peaks.get("bf16_tflops", 1958.3)
            res[prec] = entry
            del ws, G, M, X
            torch.cuda.empty_cache()
        out["precision_n16384"] = res
        del A, B
        torch.cuda.empty_cache()
    except Exception as e:  # reported, never fatal for the main line
        out["precision_n16384"] = {"error": repr(e)}

    # -- batching: 4096 systems, n ~ U{32..512}, one persistent CUDA-graph launch -----------------------
    try:
        if "batch" not in which:
            raise LookupError("not selected")
        from paper_1406_5802_gb300.batch import BatchedSolver
        sizes = W.batch_sizes(4096, 32, 512, W.SEED_BASE + 4)
        bs = BatchedSolver.synthetic(sizes, seed=W.SEED_BASE + 4, max_sweeps=40, be_tol=1e-13)
        tune = bs.tune(reps=1)
        bs.capture()
        bs.run()
        torch.cuda.synchronize()
        t0, t1 = ev(), ev()
        reps = 3
        t0.record()
        for _ in range(reps):
            bs.run()
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / reps
        berr = bs.berr.cpu().numpy()
        info = bs.info.cpu().numpy()
        ffma_peak = 152 * 128 * 2 * 2.070e9 / 1e12
        tf = bs.flops() / (ms / 1e3) / 1e12
        out["batch_4096"] = {"workload": "4096 systems, n ~ U{32..512}, A[0,0] x 1e-10, 1 RHS, FP32 GENP + FP64 "
                                         "refinement, one graph-captured persistent launch",
                             "ms_per_batch": ms, "systems_per_s": 4096 / (ms / 1e3), "tflops_fp32": tf,
                             "frac_of_fp32_fma_peak": tf / ffma_peak, "fp32_peak_tflops": ffma_peak,
                             "all_info_zero": bool(np.all(info == 0)),
                             "systems_be_le_1e-13": int(np.sum(berr <= 1e-13)), "max_berr": float(np.max(berr)),
                             "tuned": {"config": tune["config"], "ctas": tune["ctas"]}}
    except Exception as e:
        out["batch_4096"] = {"error": repr(e)}

    # -- low-rank approximation (Algorithm 6.1): n = 8192, r = l = 32, Sec. 7.2's test matrices -------------
    try:
        if "lowrank" not in which:
            raise LookupError("not selected")
        n, r = 8192, 32
        g = torch.Generator(device="cuda")
        g.manual_seed(W.SEED_BASE + 6)

        def haar(m):
            Qh, Rh = torch.linalg.qr(torch.randn(m, m, generator=g, dtype=torch.float64, device="cuda"))
            return Qh * torch.sign(torch.diagonal(Rh))[None, :]

        S, T = haar(n), haar(n)
        sig = torch.full((n,), 1e-10, dtype=torch.float64, device="cuda")
        sig[:r] = 1.0 / torch.arange(1, r + 1, dtype=torch.float64, device="cuda")
        A = (S * sig[None, :]) @ T.T
        Sr = S[:, :r].contiguous()
        del S, T
        res = {"workload": "n=8192, A = S diag(sigma) T^T with sigma_j = 1/j (j <= 32), 1e-10 beyond; l = r = 32 "
                           "(no oversampling); Q = Q(A H) by CholeskyQR2 and Z = Q^T A"}
        for kind in ("gaussian", "circulant_unitary"):
            H = rmge.lowrank_multiplier(kind, n, r, W.SEED_BASE + 6, 1)
            Q, Z, info = rmge.lowrank(kind, A, H, r)
            torch.cuda.synchronize()
            t0, t1 = ev(), ev()
            reps = 5
            t0.record()
            for _ in range(reps):
                rmge.lowrank(kind, A, H, r, Q=Q, Z=Z)
            t1.record()
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1) / reps
            # residual norms (checks, outside the timed region): rn1 = ||Q Q^T S_r - S_r||_2 exactly,
            # rn2 = ||A - Q Z||_2 by 30 power iterations
            rn1 = float(torch.linalg.matrix_norm(Q @ (Q.T @ Sr) - Sr, 2).item())
            v = torch.randn(n, 1, generator=g, dtype=torch.float64, device="cuda")
            for _ in range(30):
                w = A @ v - Q @ (Z @ v)
                v = A.T @ w - Z.T @ (Q.T @ w)
                v = v / torch.linalg.vector_norm(v)
            rn2 = float(torch.linalg.vector_norm(A @ v - Q @ (Z @ v)).item())
            flops = 2.0 * n * n * r * (1 if kind == "gaussian" else 0) + 2.0 * n * n * r + 4.0 * n * r * r
            res[kind] = {"ms": ms, "info": int(info.item()), "rn1": rn1, "rn2": rn2,
                         "fp64_tflops_gemm_part": flops / (ms / 1e3) / 1e12,
                         "note": "A H by FP64 GEMM" if kind == "gaussian" else "A H by FFT row correlation (8192-point)"}
        out["lowrank_n8192"] = res
        del A, Sr
        torch.cuda.empty_cache()
    except Exception as e:
        out["lowrank_n8192"] = {"error": repr(e)}

    # -- differentiation: 64 systems, n = 2048, FP32, forward + backward --------------------------------
    # Two forms of the same batch: FP32 factors with FP64 FGMRES sweeps (at most 3 cycles per solve: every
    # system converges in 2 forward and 1 backward), and the mixed form (emulated-FP64 factors, classical
    # FP64 sweeps).  Both return FP32 gradients of the FP64-accurate solve.
    try:
        if "grad" not in which:
            raise LookupError("not selected")
        from paper_1406_5802_gb300.autograd import rmge_solve_batched
        n, k, count = 2048, 4, 64
        g = torch.Generator(device="cuda")
        g.manual_seed(W.SEED_BASE + 5)
        As = [(4 * torch.eye(n, device="cuda") + torch.randn(n, n, generator=g, device="cuda") / n**0.5)
              .requires_grad_(True) for _ in range(count)]
        Bs = [torch.randn(n, k, generator=g, device="cuda").requires_grad_(True) for _ in range(count)]
        Ws = [torch.randn(n, k, generator=g, device="cuda") for _ in range(count)]
        res = {"workload": "64 systems, n=2048, 4 RHS, FP32, A = 4I + N(0,1)/sqrt(n), loss = sum(X*W), "
                           "forward + adjoint backward"}
        for prec, iters in (("f32", 3), ("f64x", 4)):
            def step():
                for t in As + Bs:
                    t.grad = None
                Xs = rmge_solve_batched(As, Bs, seeds=list(range(count)), prec=prec, streams=16, max_iters=iters)
                loss = sum((X * Wt).sum() for X, Wt in zip(Xs, Ws))
                loss.backward()
                return loss

            step()
            torch.cuda.synchronize()
            t0, t1 = ev(), ev()
            t0.record()
            step()
            t1.record()
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1)
            res[prec] = {"ms_per_batch": ms, "systems_per_s": count / (ms / 1e3), "max_iters": iters}
            # The same step captured once in a CUDA graph and replayed, as a training loop with fixed
            # shapes would run it: the eager step pays a host launch per kernel (hundreds per system).
            try:
                side = torch.cuda.Stream()
                side.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(side):
                    step()
                torch.cuda.current_stream().wait_stream(side)
                torch.cuda.synchronize()
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph):
                    step()
                graph.replay()
                torch.cuda.synchronize()
                t0, t1 = ev(), ev()
                t0.record()
                for _ in range(3):
                    graph.replay()
                t1.record()
                torch.cuda.synchronize()
                gms = t0.elapsed_time(t1) / 3
                res[prec]["graph_ms_per_batch"] = gms
                res[prec]["graph_systems_per_s"] = count / (gms / 1e3)
                del graph
            except Exception as e:  # report, keep the eager number
                res[prec]["graph_error"] = repr(e)[:200]
        out["grad_64x2048"] = res
    except Exception as e:
        out["grad_64x2048"] = {"error": repr(e)}
    return out


FORMS = {"f64x": ("gaussian", "f64x"), "circ_f64": ("circulant", "f64"), "circ_f64x": ("circulant", "f64x"),
         "unitary_f64x": ("circulant_unitary", "f64x"), "toeplitz_f64x": ("toeplitz", "f64x"),
         "two_sided_circ_f64x": (("circulant", "circulant"), "f64x")}
FORM_TEXT = {
    "f64x": "Gaussian G; A G and GENP's Schur updates as FP64 products emulated on the BF16 tensor cores (8 base-128 "
            "digits, 36 digit-pair MMAs, exact FP32 chunks, 64-bit fixed-point sums); pivot blocks, panels, solves, "
            "residuals and refinement in FP64",
    "circ_f64": "random circulant G (Gaussian first column) applied by FFT; GENP, solves and refinement in FP64",
    "circ_f64x": "random circulant G applied by FFT; GENP's Schur updates emulated on the BF16 tensor cores; solves and "
                 "refinement in FP64",
    "unitary_f64x": "random unitary circulant G of Ex. 5.2 (real orthogonal, unit spectrum) applied by FFT; mixed form",
    "toeplitz_f64x": "Toeplitz G = leading block of a 2n Gaussian circulant, applied by 2n-point FFTs; mixed form",
    "two_sided_circ_f64x": "random circulants on both sides (F A H y = F b, x = H y; Fact 4.1, Remark 5.1), "
                           "applied by FFT; mixed form",
}


def timed_form(rmge, A, Bm, M, X, kind, prec, args, stream, barrier, world, value_f64):
    """Whole solves (multiplier, A G, GENP, solve, refinement to the target) in one form, timed like the main
    line; the apply step is also timed on its own for the roofline of its kernel."""
    import torch

    from paper_1406_5802_gb300 import ranks
    n, k = A.shape[0], Bm.shape[1]
    two = isinstance(kind, tuple)
    if two:
        kF, kH = kind
        ws = rmge.workspace_two_sided(n, k, kF, kH, prec)
        F, H = rmge.empty_multiplier(kF, n, prec), rmge.empty_multiplier(kH, n, prec)
        T = torch.empty(n, n, dtype=torch.float64, device="cuda")
    else:
        ws = rmge.workspace(n, k, kind, prec)
        G = rmge.empty_multiplier(kind, n, prec)

    def one(i, rec=None):
        if two:
            rmge.make_multiplier(kF, n, SEED + i, 1, prec, G=F)
            rmge.make_multiplier(kH, n, SEED + i, 2, prec, G=H)
        else:
            rmge.make_multiplier(kind, n, SEED + i, 1, prec, G=G)
        if rec is not None:
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
        if two:
            rmge.apply_two_sided(kF, F, kH, H, A, prec, M=M, ws=ws, T=T)
        else:
            rmge.apply_multiplier(kind, A, G, prec, M=M, ws=ws)
        if rec is not None:
            a1.record(stream)
            rec.append((a0, a1))
        info, _ = rmge.factor(M, prec, ws=ws)
        if two:
            rmge.solve_two_sided(kF, F, kH, H, M, Bm, prec, X=X, ws=ws)
            berr, it = rmge.refine_two_sided(kF, F, kH, H, A, M, Bm, X, prec, MAX_ITERS, BE_TOL, ws=ws)
        else:
            rmge.solve(kind, M, G, Bm, prec, X=X, ws=ws)
            berr, it = rmge.refine(kind, A, M, G, Bm, X, prec, MAX_ITERS, BE_TOL, ws=ws)
        return info, berr, it

    for i in range(args.warmup):
        one(i)
    barrier()
    torch.cuda.synchronize()
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res, ev = [], []
    m0.record(stream)
    for i in range(args.steps):
        res.append(one(args.warmup + i, ev))
    m1.record(stream)
    torch.cuda.synchronize()
    ms = ranks.max_over_ranks(m0.elapsed_time(m1), world, "cuda")
    sw = [int(r[2].item()) for r in res]
    be = [float(r[1][q].item()) for r, q in zip(res, sw)]
    ok = all(int(r[0].item()) == 0 for r in res) and all(b <= BE_TOL for b in be)
    apply_ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
    val = ranks.whole_job_rate(args.steps, world, ms / 1e3)
    out = {"form": FORM_TEXT[args_form_key(kind, prec)], "value": val, "unit": "solves/s",
           "ms_per_step": ms / args.steps, "all_steps_be_le_1e-13": ok, "max_berr": max(be),
           "mean_sweeps": sum(sw) / len(sw), "apply_ms": apply_ms, "speedup_vs_f64": val / value_f64,
           "tflops": flops_per_solve(n, k, sum(sw) / len(sw)) * val / 1e12}
    if kind == "gaussian" and prec == "f64x":
        pairs = 36  # base-128 digit pairs kept by the emulated FP64 product (8 digits per entry)
        out["roofline"] = {"kernel": "oz_gemm_kernel (M = A G)", "bound": "tensor",
                           "achieved": pairs * 2 * n**3 / (apply_ms / 1e3) / 1e12, "peak": None,
                           "unit": "TFLOP/s (BF16 MMA)", "frac": None,
                           "traffic": OZ_AG_TRAFFIC_BYTES if n == N_SYS else None,
                           "algorithmic_bytes": 3 * n * n * 8 + 2 * 8 * n * n * 2}
    del ws
    return out


def args_form_key(kind, prec):
    for key, (fk, fp) in FORMS.items():
        if fk == kind and fp == prec:
            return key
    return "f64"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rmge", choices=["rmge", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other measured workloads")
    ap.add_argument("--extras", default="precision,batch,grad,lowrank",
                    help="comma list of the other workloads (precision, batch, grad, lowrank)")
    ap.add_argument("--forms", default="f64x,circ_f64,circ_f64x,unitary_f64x,toeplitz_f64x,two_sided_circ_f64x",
                    help="comma list of the other forms timed on the same inputs (f64x, circ_f64, circ_f64x, "
                         "unitary_f64x, toeplitz_f64x, two_sided_circ_f64x; "
                         "'none' for the main line only)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1406_5802_gb300 import ranks
    from paper_1406_5802_gb300 import rmge
    from paper_1406_5802_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_1406_5802_gb300 import build as B
    if rank == 0:
        B.build()
    barrier()
    rmge.load_library()

    n, k = N_SYS, K_RHS
    A_np, B_np = W.orthogonal_factor_system(n, k, SIGMA_MIN, seed=ranks.system_seed(SEED, rank))
    A = torch.as_tensor(A_np).cuda()
    Bm = torch.as_tensor(B_np).cuda()
    kind, prec = "gaussian", "f64"
    ws = rmge.workspace(n, k, kind, prec)
    G = rmge.empty_multiplier(kind, n, prec)
    M = torch.empty(n, n, dtype=torch.float64, device="cuda")
    X = torch.empty(n, k, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    ev_apply = []

    def step(i, record=False):
        rmge.make_multiplier(kind, n, SEED + i, 1, prec, G=G)
        if record:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        rmge.apply_multiplier(kind, A, G, prec, M=M, ws=ws)
        if record:
            e1.record(stream)
            ev_apply.append((e0, e1))
        info, growth = rmge.factor(M, prec, ws=ws)
        rmge.solve(kind, M, G, Bm, prec, X=X, ws=ws)
        berr, iters = rmge.refine(kind, A, M, G, Bm, X, prec, MAX_ITERS, BE_TOL, ws=ws)
        return info, berr, iters

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    stop = threading.Event()
    clk = []
    th = threading.Thread(target=sample_clocks, args=(stop, clk), daemon=True)
    th.start()
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    results = []
    launches0 = rmge.kernel_launches()
    for i in range(args.steps):
        results.append(step(args.warmup + i, record=True))
    launches = rmge.kernel_launches() - launches0
    t1.record(stream)
    torch.cuda.synchronize()
    stop.set()
    th.join(timeout=2)
    barrier()
    ms = t0.elapsed_time(t1)
    ms_max = ranks.max_over_ranks(ms, world, "cuda")  # the whole job lasts as long as its slowest rank

    # every timed solve must have met the accuracy target
    infos = [int(r[0].item()) for r in results]
    sweeps = [int(r[2].item()) for r in results]
    bes = [float(r[1][s].item()) for r, s in zip(results, sweeps)]
    ok = all(i == 0 for i in infos) and all(b <= BE_TOL for b in bes)
    # independent check of the last solve by the oracle's compensated residual (rank 0)
    be_oracle = None
    if rank == 0:
        from oracle import oracle as orc
        orc.set_threads(os.cpu_count() or 1)
        be_oracle = orc.backward_error(A.cpu().numpy(), X.cpu().numpy(), Bm.cpu().numpy())

    value = ranks.whole_job_rate(args.steps, world, ms_max / 1e3)
    mean_sweeps = sum(sweeps) / len(sweeps)
    flops = flops_per_solve(n, k, mean_sweeps)
    apply_ms = sum(a.elapsed_time(b) for a, b in ev_apply) / len(ev_apply)
    achieved = (2 * n**3 - n**2) / (apply_ms / 1e3) / 1e12

    # the other forms on the same inputs and the same accuracy target: the mixed form (A G and GENP's
    # Schur updates as FP64 products emulated on the BF16 tensor cores, RMGE_F64X_TC) and the random
    # circulant multiplier applied by FFT (Sec. 5), in FP64 and in the mixed form
    forms = {}
    wanted = [f for f in args.forms.split(",") if f and f != "none"]
    for name in wanted:
        fkind, fprec = FORMS[name]
        try:
            forms[name] = timed_form(rmge, A, Bm, M, X, fkind, fprec, args, stream, barrier, world, value)
        except Exception as e:  # reported, never fatal for the main line
            forms[name] = {"error": repr(e)}

    # end to end through the public API with host buffers: H2D of A and B, D2H of X and berr each step
    A_h = A.cpu().pin_memory()
    B_h = Bm.cpu().pin_memory()
    X_h = torch.empty(n, k, dtype=torch.float64).pin_memory()
    be_h = torch.empty(MAX_ITERS + 1, dtype=torch.float64).pin_memory()
    A_d = torch.empty_like(A)
    B_d = torch.empty_like(Bm)
    barrier()
    torch.cuda.synchronize()
    te = time.perf_counter()
    for i in range(args.steps):
        A_d.copy_(A_h, non_blocking=True)
        B_d.copy_(B_h, non_blocking=True)
        rmge.make_multiplier(kind, n, SEED + i, 1, prec, G=G)
        rmge.apply_multiplier(kind, A_d, G, prec, M=M, ws=ws)
        rmge.factor(M, prec, ws=ws)
        rmge.solve(kind, M, G, B_d, prec, X=X, ws=ws)
        berr, _ = rmge.refine(kind, A_d, M, G, B_d, X, prec, MAX_ITERS, BE_TOL, ws=ws)
        X_h.copy_(X, non_blocking=True)
        be_h.copy_(berr, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - te
    e2e_value = ranks.whole_job_rate(args.steps, world, ranks.max_over_ranks(e2e_s, world, "cuda"))

    if rank == 0:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        cpu = None
        if not args.no_cpu_baseline:
            cores = os.cpu_count() or 1
            dt, _ = cpu_oracle_solve(A.cpu().numpy(), Bm.cpu().numpy(), G.cpu().numpy(), cores)
            cpu = {"value": 1.0 / dt, "unit": "solves/s", "cores": cores, "kind": "oracle",
                   "sample": "one full n=4096, 16-RHS oracle solve (plain C FP64, OpenMP over rows) with the "
                             "same A, B and G as the last timed GPU step"}
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "randomized GENP solve, n=4096, 16 RHS, FP64, Gaussian multiplier",
                       "n": n, "nrhs": k, "sigma": "log-spaced 1..1e-6", "precision": "f64",
                       "l2": "inputs larger than L2 (A, G, M 134 MB each)", "replicas": world},
            "tflops": flops * value / 1e12,
            "accuracy": {"all_steps_be_le_1e-13": ok, "max_berr": max(bes), "mean_sweeps": mean_sweeps,
                         "oracle_berr_last": be_oracle},
            "roofline": {"kernel": "gemm_kernel (M = A G, FP64 DFMA)", "bound": "alu", "achieved": achieved,
                         "peak": FP64_ALU_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_ALU_PEAK_TFLOPS,
                         "traffic": AG_TRAFFIC_BYTES,
                         "algorithmic_bytes": 3 * n * n * 8,
                         "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.070 GHz (FP64 is not in "
                                        "MEASURED_PEAKS.json)",
                         "apply_ms": apply_ms},
            "e2e": {"value": e2e_value, "unit": "solves/s",
                    "h2d_bytes_per_step": (A.numel() + Bm.numel()) * 8,
                    "d2h_bytes_per_step": (X.numel() + MAX_ITERS + 1) * 8},
            "gpu_launches": launches,
            "clocks": clocks_summary(clk),
            "cpu_baseline": cpu,
            "hbm_gbs_measured_peak": peaks.get("hbm_gbs"),
            "forms": forms,
        }
        for f in forms.values():
            if isinstance(f, dict) and isinstance(f.get("roofline"), dict) and f["roofline"].get("unit", "").startswith("TFLOP/s (BF16"):
                pk = peaks.get("bf16_tflops", 1958.3)
                f["roofline"]["peak"] = pk
                f["roofline"]["frac"] = f["roofline"]["achieved"] / pk
                f["roofline"]["peak_source"] = "MEASURED_PEAKS.json bf16_tflops (burst), of measured"
        if not args.no_extras:
            sel = tuple(x for x in args.extras.split(",") if x)
            line["extras"] = {k: v for k, v in extra_workloads(W, rmge, peaks, sel).items()
                              if not (isinstance(v, dict) and v.get("error") == repr(LookupError("not selected")))}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
