"""Learned warm start for the Jacobi Poisson solve: data, training, evaluation.

    python -m paper_2310_01882_b300.warmstart [--n 128] [--train 200] [--test 20]
        [--epochs 30] [--batch 4] [--lr 1e-3] [--together K] [--kinds LIST] [--out DIR]

Pairs (f, u*): f a k^-3 Gaussian random field (seeds 10000+i for training,
20000+i held out), u* from plain FP64 Jacobi (stencil_jacobi_sweep) from zero
until the FP64 relative residual (stencil_residual) is at most 1e-8.  The
net (wsnet_*, 4 levels 16-32-64-64) is trained with Adam and a cosine
learning-rate decay; on the held-out fields the sweeps and wall time to
relative residual 1e-8 are measured for a zero start and for the warm start,
with plain FP64 Jacobi and with the mixed-precision solve
(stencil_batch_solve, FP32 inner storage).  The residual computed in FP64 is
the arbiter throughout.  The warm start's own residual is recorded; the
"selected" figures use it only when, after `check_sweeps` plain sweeps from
each start, its residual is below the zero start's (the fallback is plain
Jacobi from zero).  With --together K, K held-out fields are also solved as
one job (throughput): plain FP64 Jacobi over several streams against the
batch solve with FP32 and BF16 inner storage, from zero and warm starts.

Host-side orchestration only: every step runs in the library's kernels.
"""
import argparse
import json
import math
import os
import time

import numpy as np

from . import inputs
from . import stencil as S

CHANNELS = [16, 32, 64, 64]
RTOL = 1e-8
# The network trained on 2000 (f, u*) pairs of 128^3 (seeds 10000..11999),
# 30 epochs: its parameters in wsnet_load's parameters-only format.
TRAINED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "wsnet_128cubed_2000pairs.wsnet")


def save_params_only(path, levels, channels, n, params):
    """Write parameters in the parameters-only file format wsnet_load reads
    (magic "WSNET01", int32 levels, int32 channels[levels], int32 n, int64
    count, FP32 parameters; little endian); loading it starts the optimiser
    afresh."""
    import struct
    params = np.ascontiguousarray(params, dtype="<f4")
    with open(path + ".tmp", "wb") as fh:
        fh.write(b"WSNET01\x00")
        fh.write(struct.pack("<i", levels))
        fh.write(struct.pack(f"<{levels}i", *channels))
        fh.write(struct.pack("<iq", n, params.size))
        fh.write(params.tobytes())
    os.replace(path + ".tmp", path)


def trained_net(n=128):
    """The committed trained network (for 128^3 grids)."""
    net = S.WsNet(len(CHANNELS), CHANNELS, n, seed=1)
    S.wsnet_load(net, TRAINED)
    return net


def warm_starts(net, ctx, fs, h, norms, tmp, check_sweeps=50):
    """Warm starts for the F64 source Fields fs: the network's output where,
    after `check_sweeps` plain FP64 Jacobi sweeps from it and from zero, its
    FP64 relative residual is the smaller, else None (the fallback: plain
    Jacobi from zero).  The output's own residual is no guide: its error is
    mostly high-frequency, which the first sweeps remove, so it starts above
    the zero start's and ends far below.  tmp: an F64 Field of the same
    extents (scratch).  Returns (starts, residuals after the check from the
    warm start, from zero); the caller times it."""
    n = fs[0].nx
    starts, rw, rz = [], [], []
    for f in fs:
        u = S.Field(n, n, n)
        S.wsnet_infer(net, f, u)
        start = u.storage.clone()
        rels = []
        for v in (u, S.Field(n, n, n)):
            S.stencil_jacobi_sweep(ctx, v, tmp, f, None, h, check_sweeps, 0, S.SWEEP_AUTO)
            S.stencil_residual(ctx, v, f, h, norms)
            nrm = norms.cpu().numpy()
            rels.append(float(nrm[0] / nrm[1]))
        rw.append(rels[0])
        rz.append(rels[1])
        starts.append(start if rels[0] < rels[1] else None)
    return starts, rw, rz


class Solver:
    """Plain FP64 Jacobi (or red-black) on one grid size, one context per
    stream.  The sweep shape and pass length are the library's compiled
    configuration that finishes a chunk of sweeps soonest when run the way
    the solve runs them: on one stream for a single problem, on every stream
    at once for several (tuned once per case on seeded problems of this
    size)."""

    def __init__(self, n, streams=1, tune=True):
        import torch
        self.n = n
        self.h = 1.0 / (n + 1)
        self.ctxs = [S.Context(0) for _ in range(streams)]
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.tmp = [S.Field(n, n, n) for _ in range(streams)]
        self.work = [S.Field(n, n, n) for _ in range(streams)]
        self.norms = torch.zeros((streams, 2), dtype=torch.float64, device="cuda")
        self.tune = tune
        self.choice = {}   # (redblack, concurrent streams) -> (sweeps per pass, configuration index)
        self.tune_log = {}

    def _pick(self, redblack, k, chunk):
        """Time every compiled FP64 (resident fixed point) configuration on
        k concurrent seeded problems, `chunk` sweeps each; keep the fastest."""
        import torch
        key = (redblack, k)
        if key in self.choice:
            return self.choice[key]
        if not self.tune:
            self.choice[key] = (1, 0)
            return self.choice[key]
        n = self.n
        us = [S.Field.from_numpy(inputs.uniform(n, n, n, seed=3 + j)) for j in range(k)]
        fs = make_fields(n, [2 + j for j in range(k)])
        if redblack:
            cands = [(1, i) for i in range(S.stencil_redblack_config_count(S.F64, S.SWEEP_AUTO, True, 1))]
        else:
            cands = [(T, i) for T in (1, 2) for i in range(S.stencil_sweep_config_count(S.F64, S.SWEEP_AUTO, True, T))]
        sweep = S.stencil_redblack_sweep if redblack else S.stencil_jacobi_sweep
        best, log = None, []
        for T, i in cands:
            for c in self.ctxs[:k]:
                if redblack:
                    S.stencil_redblack_config_select(c, S.F64, S.SWEEP_AUTO, True, T, i)
                else:
                    S.stencil_sweep_config_select(c, S.F64, S.SWEEP_AUTO, True, T, i)
            times = []
            for rep in range(2):  # the first round warms up
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for j in range(k):
                    sweep(self.ctxs[j], us[j], self.tmp[j], fs[j], self.work[j], self.h, chunk, T, S.SWEEP_AUTO,
                          stream=self.streams[j])
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
            log.append((T, i, times[-1]))
            if best is None or times[-1] < best[2]:
                best = (T, i, times[-1])
        self.choice[key] = (best[0], best[1])
        self.tune_log[key] = log
        return self.choice[key]

    def solve(self, us, fs, chunk=1000, max_sweeps=2_000_000, redblack=False):
        """Sweep every u (F64 Fields, in place) until its relative residual is
        <= RTOL, checking every `chunk` sweeps.  The streams work through the
        instances as a queue: a stream whose instance has finished takes the
        next one.  Returns per-instance (sweeps, rel)."""
        import torch
        out = [None] * len(us)
        k = len(self.streams)
        T, idx = self._pick(redblack, min(k, len(us)), chunk)
        for c in self.ctxs:
            if redblack:
                S.stencil_redblack_config_select(c, S.F64, S.SWEEP_AUTO, True, T, idx)
            else:
                S.stencil_sweep_config_select(c, S.F64, S.SWEEP_AUTO, True, T, idx)
        queue = list(range(len(us)))[::-1]
        slot = [None] * k
        sweeps = [0] * len(us)
        while True:
            for j in range(k):
                if slot[j] is None and queue:
                    slot[j] = queue.pop()
            if all(i is None for i in slot):
                return out
            for j, i in enumerate(slot):
                if i is not None:
                    S.stencil_residual(self.ctxs[j], us[i], fs[i], self.h, self.norms[j], stream=self.streams[j])
            torch.cuda.synchronize()
            nrm = self.norms.cpu().numpy()
            for j, i in enumerate(slot):
                if i is None:
                    continue
                rel = nrm[j, 0] / nrm[j, 1]
                if rel <= RTOL or sweeps[i] >= max_sweeps:
                    out[i] = (sweeps[i], float(rel))
                    slot[j] = None
                    continue
                sweep = S.stencil_redblack_sweep if redblack else S.stencil_jacobi_sweep
                sweep(self.ctxs[j], us[i], self.tmp[j], fs[i], self.work[j], self.h, chunk, T, S.SWEEP_AUTO,
                      stream=self.streams[j])
                sweeps[i] += chunk


def make_fields(n, seeds, workers=None):
    """Device Fields of the k^-3 GRFs for `seeds`, in seed order; the host
    transforms run on several threads, a few fields ahead of the copies."""
    from concurrent.futures import ThreadPoolExecutor
    workers = workers or max(1, min(16, len(os.sched_getaffinity(0))))
    out = []
    with ThreadPoolExecutor(workers) as ex:
        for b in range(0, len(seeds), 4 * workers):
            chunk = seeds[b:b + 4 * workers]
            out += [S.Field.from_numpy(a) for a in ex.map(lambda s: inputs.grf(n, seed=s), chunk)]
    return out


def generate_pairs(solver, seeds):
    """(f, u*) Field pairs for the given GRF seeds (u* from plain FP64 Jacobi)."""
    n = solver.n
    fs = make_fields(n, seeds)
    us = [S.Field(n, n, n) for _ in seeds]
    info = solver.solve(us, fs)
    return fs, us, info


def train(net, fs, us, epochs, batch, lr0, seed=0, log=None, ckpt_dir=None, stop_after=None):
    """Adam with a cosine decay from lr0 to lr0/20 over all steps.  With
    ckpt_dir, a checkpoint is written after every epoch (the net with its
    Adam state, wsnet_save; the epoch, step count, loss history and the
    batch-order generator's state) and, if one is there already, training
    resumes after its epoch exactly as if it had not stopped.  stop_after:
    return after that many epochs (of `epochs`) in this call."""
    rng = np.random.default_rng(seed)
    steps = epochs * max(1, len(fs) // batch)
    hist = []
    step = 0
    ep0 = 0
    state_path = os.path.join(ckpt_dir, "train_state.json") if ckpt_dir else None
    if state_path and os.path.exists(state_path):
        with open(state_path) as fh:
            st = json.load(fh)
        S.wsnet_load(net, os.path.join(ckpt_dir, "wsnet.ckpt"))
        rng.bit_generator.state = st["rng"]
        hist, step, ep0 = st["hist"], st["step"], st["epoch"] + 1
    for ep in range(ep0, epochs if stop_after is None else min(epochs, stop_after)):
        order = rng.permutation(len(fs))
        losses = []
        for b in range(0, len(fs) - batch + 1, batch):
            lr = lr0 * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * step / max(1, steps))))
            sel = order[b:b + batch]
            losses.append(S.wsnet_train_step(net, [fs[i] for i in sel], [us[i] for i in sel], lr))
            step += 1
        hist.append(float(np.mean(losses)))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
        if ckpt_dir:
            os.makedirs(ckpt_dir, exist_ok=True)
            S.wsnet_save(net, os.path.join(ckpt_dir, "wsnet.ckpt.tmp"))
            os.replace(os.path.join(ckpt_dir, "wsnet.ckpt.tmp"), os.path.join(ckpt_dir, "wsnet.ckpt"))
            with open(state_path + ".tmp", "w") as fh:
                json.dump({"epoch": ep, "step": step, "hist": hist, "rng": rng.bit_generator.state}, fh)
            os.replace(state_path + ".tmp", state_path)
    return hist


def evaluate(net, solver, seeds, chunk=200, check_sweeps=50):
    """Sweeps / seconds to RTOL from a zero start and from the warm start,
    with plain FP64 Jacobi and with the mixed-precision batch solve."""
    import torch
    n, h = solver.n, solver.h
    ctx = solver.ctxs[0]
    rows = []
    for s in seeds:
        f_np = inputs.grf(n, seed=s)
        f = S.Field.from_numpy(f_np)
        r = {"seed": s}
        # warm start (inference timed), checked by its FP64 residual
        u_w = S.Field(n, n, n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.wsnet_infer(net, f, u_w)
        S.stencil_residual(ctx, u_w, f, h, solver.norms[0])
        torch.cuda.synchronize()
        r["infer_s"] = time.perf_counter() - t0
        nrm = solver.norms[0].cpu().numpy()
        r["warm_rel0"] = float(nrm[0] / nrm[1])
        warm0 = u_w.storage.clone()
        for name, start in (("zero", None), ("warm", warm0)):
            u = S.Field(n, n, n)
            if start is not None:
                u.storage.copy_(start)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            (sw, rel), = solver.solve([u], [f], chunk=chunk)
            torch.cuda.synchronize()
            r[f"fp64_{name}"] = {"sweeps": sw, "seconds": time.perf_counter() - t0, "rel": rel}
            u = S.Field(n, n, n)
            if start is not None:
                u.storage.copy_(start)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = S.stencil_batch_solve(ctx, [u], [f], [h], RTOL, inner_dtype=S.F32, sweeps_per_cycle=400)
            torch.cuda.synchronize()
            r[f"mixed_{name}"] = {"sweeps": res[0]["sweeps"], "seconds": time.perf_counter() - t0,
                                  "rel": res[0]["rel_residual"], "status": res[0]["status"]}
        # check: residual after check_sweeps plain sweeps from each start
        rels = {}
        for name, start in (("zero", None), ("warm", warm0)):
            u = S.Field(n, n, n)
            if start is not None:
                u.storage.copy_(start)
            S.stencil_jacobi_sweep(ctx, u, solver.tmp[0], f, None, h, check_sweeps, 0, S.SWEEP_AUTO)
            S.stencil_residual(ctx, u, f, h, solver.norms[0])
            nrm = solver.norms[0].cpu().numpy()
            rels[name] = float(nrm[0] / nrm[1])
        r["check_rel"] = rels
        r["fallback"] = not (rels["warm"] < rels["zero"])
        rows.append(r)
    return rows


def solve_together(solver, fs, starts, kind, chunk=200, sweeps_per_cycle=400):
    """Bring every field to RTOL together (throughput: the fields are solved
    as one job) and time it.  kind "fp64": plain FP64 Jacobi on the
    solver's streams, residual checked every `chunk` sweeps ("fp64rb":
    red-black Gauss-Seidel); "f32"/"bf16": stencil_batch_solve with that
    inner storage, every active instance in one persistent launch per pass
    ("f32rb": red-black inner sweeps).  starts: list of None (zero) or F64
    storage tensors to copy.  Returns (seconds, sweeps list, max rel, ok)."""
    import torch
    n, h = solver.n, solver.h
    us = []
    for st in starts:
        u = S.Field(n, n, n)
        if st is not None:
            u.storage.copy_(st)
        us.append(u)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if kind in ("fp64", "fp64rb"):
        info = solver.solve(us, fs, chunk=chunk, redblack=(kind == "fp64rb"))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        sweeps = [sw for sw, _ in info]
        rels = [rel for _, rel in info]
        ok = all(r <= RTOL for r in rels)
    else:
        inner = S.BF16 if kind.startswith("bf16") else S.F32
        res = S.stencil_batch_solve(solver.ctxs[0], us, fs, [h] * len(us), RTOL, inner_dtype=inner,
                                    sweeps_per_cycle=sweeps_per_cycle, smoother=int(kind.endswith("rb")))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        sweeps = [r["sweeps"] for r in res]
        rels = [r["rel_residual"] for r in res]
        ok = all(r["status"] == 0 and r["rel_residual"] <= RTOL for r in res)
    # the FP64 residual of every returned u decides
    worst = 0.0
    for u, f in zip(us, fs):
        S.stencil_residual(solver.ctxs[0], u, f, h, solver.norms[0])
        nrm = solver.norms[0].cpu().numpy()
        worst = max(worst, float(nrm[0] / nrm[1]))
    return dt, sweeps, worst, ok and worst <= RTOL


def evaluate_together(net, solver, seeds, kinds=("fp64", "f32", "bf16")):
    """Time to bring ALL the held-out fields to RTOL as one job, from zero
    starts and from warm starts (inference of every field included)."""
    import torch
    n = solver.n
    fs = make_fields(n, seeds)
    warm = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if net is not None:
        for f in fs:
            u = S.Field(n, n, n)
            S.wsnet_infer(net, f, u)
            warm.append(u.storage)
    torch.cuda.synchronize()
    infer_s = time.perf_counter() - t0
    out = {"fields": len(seeds), "infer_seconds": infer_s}
    for start in (("zero", "warm") if net is not None else ("zero",)):
        starts = [None] * len(fs) if start == "zero" else warm
        for kind in kinds:
            dt, sweeps, worst, ok = solve_together(solver, fs, starts, kind)
            if start == "warm":
                dt += infer_s
            out[f"{kind}_{start}"] = {"seconds": dt, "sweeps_median": float(np.median(sweeps)),
                                      "sweeps_total": int(np.sum(sweeps)), "worst_rel": worst, "ok": ok}
    base = out["fp64_zero"]["seconds"]
    out["speedup_vs_fp64_zero"] = {k: base / v["seconds"] for k, v in out.items()
                                   if isinstance(v, dict) and "seconds" in v and k != "fp64_zero"}
    return out


def summarise(rows):
    def med(key, field):
        return float(np.median([r[key][field] for r in rows]))
    out = {k: {"sweeps_median": med(k, "sweeps"), "seconds_median": med(k, "seconds")}
           for k in ("fp64_zero", "fp64_warm", "mixed_zero", "mixed_warm")}
    inf = float(np.median([r["infer_s"] for r in rows]))
    base = out["fp64_zero"]["seconds_median"]
    out["infer_seconds_median"] = inf
    out["speedup_vs_fp64_zero"] = {k: base / (out[k]["seconds_median"] + (inf if "warm" in k else 0.0))
                                   for k in ("fp64_warm", "mixed_zero", "mixed_warm")}
    out["warm_rel0_median"] = float(np.median([r["warm_rel0"] for r in rows]))
    out["fallbacks"] = int(sum(1 for r in rows if r.get("fallback")))
    # with the fallback applied: the warm start only where the check accepted it
    sel = []
    for r in rows:
        k = "mixed_zero" if r.get("fallback") else "mixed_warm"
        sel.append(r[k]["seconds"] + (0.0 if r.get("fallback") else r["infer_s"]))
    out["selected_mixed_seconds_median"] = float(np.median(sel))
    out["speedup_selected_mixed_vs_fp64_zero"] = base / float(np.median(sel))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--train", type=int, default=200)
    ap.add_argument("--test", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--streams", type=int, default=8)
    ap.add_argument("--load", default=None,
                    help="evaluate saved parameters (.npy, or a wsnet file such as the committed TRAINED) instead of training")
    ap.add_argument("--together", type=int, default=0,
                    help="also time solving this many held-out fields as one job")
    ap.add_argument("--kinds", default="fp64,f32,bf16",
                    help="solvers of the --together comparison (fp64, fp64rb, f32, f32rb, bf16)")
    ap.add_argument("--checkpoint", default=None,
                    help="directory for per-epoch training checkpoints (resumes from one found there)")
    ap.add_argument("--out", default=".")
    args = ap.parse_args()
    import torch
    log = lambda m: print(m, flush=True)  # noqa: E731
    solver = Solver(args.n, streams=args.streams)
    net = S.WsNet(len(CHANNELS), CHANNELS, args.n, seed=1)
    gen_s = train_s = 0.0
    hist = []
    if args.load:
        if args.load.endswith(".npy"):
            net.set_params(np.load(args.load))
        else:  # a wsnet_save / save_params_only file (e.g. TRAINED)
            S.wsnet_load(net, args.load)
        args.train = args.epochs = 0
    else:
        t0 = time.perf_counter()
        fs, us, info = generate_pairs(solver, [10000 + i for i in range(args.train)])
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
        log(f"generated {args.train} pairs in {gen_s:.1f} s; sweeps median {np.median([s for s, _ in info])}")
        t0 = time.perf_counter()
        hist = train(net, fs, us, args.epochs, args.batch, args.lr, log=log, ckpt_dir=args.checkpoint)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        del fs, us
        np.save(os.path.join(args.out, "wsnet_params.npy"), net.get_params())
        save_params_only(os.path.join(args.out, "wsnet_params.wsnet"), len(CHANNELS), CHANNELS, args.n,
                         net.get_params())
    rows = evaluate(net, solver, [20000 + i for i in range(args.test)])
    summary = summarise(rows)
    log(json.dumps(summary))
    together = None
    if args.together:
        together = evaluate_together(net, solver, [20000 + i for i in range(args.together)],
                                     kinds=tuple(args.kinds.split(",")))
        log(json.dumps(together))
    result = {"n": args.n, "train_pairs": args.train, "test_fields": args.test, "epochs": args.epochs,
              "batch": args.batch, "lr": args.lr, "gen_seconds": gen_s, "train_seconds": train_s,
              "loss_history": hist, "summary": summary, "rows": rows, "together": together}
    with open(os.path.join(args.out, "warmstart.json"), "w") as fh:
        json.dump(result, fh, indent=1)


if __name__ == "__main__":
    main()
