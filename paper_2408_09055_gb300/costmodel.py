"""Learned kernel-cost model: timing data from this simulator on the GPU,
training with the library's own kernels, save/load.

Every sample is one kernel of the kind the planners emit, timed as the
library executes it on a resident 30-qubit state:

* shared-memory samples: a random subcircuit (an active set of 1..13 of the
  30 qubits -- the planner's range -- and 1..64 gates inside it, drawn from
  the mixed-circuit gate set or, for every other sample, from all ten gate
  types), planned as a single shared-memory kernel and compiled to its
  specialised form;
* fused samples: a random subcircuit on 1..6 qubits applied as one fused
  unitary in the requested precision;
* planner-shaped samples (a fraction of the count): kernels of analytic
  Kernelize plans of freshly seeded 30-qubit mixed and entangling circuits
  (seeds distinct from any benchmark seed), each timed alone -- the kernels
  the planner actually weighs, which random subcircuits rarely resemble
  (dozens of dense gates on 11..14 qubits).

Features come from ``qs_kernel_features`` of the kernel as planned; the
target is ln(microseconds).  Training runs ``qs_mlp_train_step`` (the
library's FP32 forward/backward/Adam kernels) on mini-batches; inference in
the planners uses the BF16 weights.  This module only marshals arguments and
orchestrates; all arithmetic runs in libqsim's kernels.
"""
from __future__ import annotations

import concurrent.futures as cf
import json
import math
import os
import time

import numpy as np

from . import qsim as Q

PKG = os.path.dirname(os.path.abspath(__file__))
MODEL_PATH = os.path.join(PKG, "data", "costmodel_gb300.npz")
N_REF = 30  # state size the timings are taken on


def _sample_specs(n, count, seed, fused_fraction, precision, max_active=13):
    from synth import circuits as C
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        sub_seed = int(rng.integers(0, 2 ** 62))
        fused = rng.uniform() < fused_fraction
        gate_set = C.ALL_TYPES if i % 2 else C.MIXED_SET
        if fused:
            g, _ = C.random_subcircuit(n, seed=sub_seed, max_active=6, gate_set=gate_set)
            cost = Q.default_cost_table()
            for k in range(16):
                cost.fuse_cost[k] = 1.0
            opts = Q.default_opts(algo=Q.QS_ALGO_ORDERED, fuse_kmax=6, precision=precision, cost=cost)
        else:
            g, _ = C.random_subcircuit(n, seed=sub_seed, max_active=max_active, gate_set=gate_set)
            opts = Q.default_opts(algo=Q.QS_ALGO_ORDERED, fuse_kmax=0, shm_max_active=14)
        specs.append((g, opts, opts.cost))
    return specs


def _workload_specs(n, count, seed):
    """Kernels of analytic Kernelize plans of seeded workload circuits, as
    single-kernel specs (greedy packing of the kernel's gates, which keeps
    them in one shared-memory kernel)."""
    from synth import circuits as C
    rng = np.random.default_rng(seed + 7919)
    specs = []
    while len(specs) < count:
        wseed = 10_000 + int(rng.integers(0, 1 << 30))
        if rng.uniform() < 0.5:
            g = C.mixed_circuit(n, 1200, wseed)
        else:
            g = C.entangling_circuit(n, 10, wseed)
        smax = int(rng.integers(11, 15))
        plan = Q.Plan(n, g, Q.default_opts(algo=Q.QS_ALGO_KERNELIZE, fuse_kmax=0, shm_max_active=smax,
                                           shm_variant=2))
        nk = plan.stats().num_kernels
        for k in rng.permutation(nk)[:max(1, nk // 4)]:
            sub = g[plan.kernel_gates(int(k))]
            opts = Q.default_opts(algo=Q.QS_ALGO_GREEDY, fuse_kmax=0, shm_max_active=14)
            specs.append((sub, opts, opts.cost))
            if len(specs) >= count:
                break
    return specs


def _build(n, spec):
    g, opts, _keep = spec
    plan = Q.Plan(n, g, opts)
    if plan.stats().num_kernels != 1:
        return None
    return plan


def generate(n=N_REF, count=4096, seed=0, fused_fraction=0.25, precision=Q.QS_PREC_TF32X3,
             reps=3, batch=256, threads=None, stream=None, log=print, max_active=13,
             workload_fraction=0.2):
    """Times `count` random kernels; returns (X [count x F], y = ln(us), meta)."""
    import torch
    threads = threads or os.cpu_count() or 4
    nw = int(round(workload_fraction * count))
    specs = _sample_specs(n, count - nw, seed, fused_fraction, precision, max_active)
    specs += _workload_specs(n, nw, seed)
    buf = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    st = Q.State(n, buf.data_ptr())
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    st.set_zero(s)
    t0 = time.time()
    X, y, kinds = _time_specs(n, specs, reps, st, s, threads)
    if log:
        log(f"timed {len(y)} kernels in {time.time() - t0:.0f} s")
    meta = {"n": n, "count": len(y), "seed": seed, "fused_fraction": fused_fraction, "max_active": max_active,
            "workload_fraction": workload_fraction,
            "precision": int(precision), "reps": reps, "seconds": time.time() - t0,
            "fused_samples": int(sum(1 for k in kinds if k == Q.QS_KERNEL_FUSED))}
    return np.asarray(X, dtype=np.float32), np.asarray(y, dtype=np.float32), meta


def _time_specs(n, specs, reps, st, s, threads, log=None):
    """Plans every spec as one kernel and times it; returns (X, y, kinds)."""
    X, y, kinds = [], [], []
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for b0 in range(0, len(specs), 256):
            part = specs[b0:b0 + 256]
            plans = list(ex.map(lambda sp: _build(n, sp), part))
            for sp, plan in zip(part, plans):
                if plan is None:
                    continue
                d = plan.kernel(0)
                ids = plan.kernel_gates(0)
                st.run(plan, s)  # warm-up: uploads and loads the kernel
                timer = Q.Timer(plan, reps)
                for _ in range(reps):
                    st.run_timed(plan, timer, s)
                ms, runs = timer.read()
                X.append(Q.qs_kernel_features(n, sp[0][ids], d.type, d.qubit_mask))
                y.append(math.log(ms[0] / runs * 1e3))
                kinds.append(d.type)
            del plans
    return X, y, kinds


def refine(net, X, y, n=N_REF, rounds=2, circuits=6, seed=0, precision=Q.QS_PREC_TF32X3, reps=3,
           epochs=300, threads=None, log=print, weight=4, entangling_share=0.67, tau=0.5, ensemble=1,
           contrast=False, shm_max=12):
    """Active refinement: plan freshly seeded workload circuits with the
    learned cost (Kernelize, fused kernels in `precision`), time exactly the
    kernels those plans chose, add them to the data and retrain.  A planner
    that minimises a learned cost steers towards kernels the model
    underestimates; timing its own choices corrects those regions.  With
    `contrast` the analytic plans' kernels of the same circuits are timed too,
    so the model also learns the alternative it is weighed against."""
    import torch
    from synth import circuits as C
    threads = threads or os.cpu_count() or 4
    rng = np.random.default_rng(seed + 104729)
    buf = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    st = Q.State(n, buf.data_ptr())
    s = torch.cuda.current_stream().cuda_stream
    st.set_zero(s)
    fcost = Q.default_cost_table()
    for k in range(16):
        fcost.fuse_cost[k] = 1.0
    metrics, history = {}, []
    base = split(len(y), seed)
    Xr = np.zeros((0, X.shape[1]), dtype=np.float32)  # refinement samples
    yr = np.zeros(0, dtype=np.float32)
    for r in range(rounds):
        specs = []
        for _ in range(circuits):
            wseed = 20_000 + int(rng.integers(0, 1 << 30))
            ent = rng.uniform() < entangling_share
            g = C.entangling_circuit(n, 10, wseed) if ent else C.mixed_circuit(n, 1200, wseed)
            plans = [Q.Plan(n, g, Q.default_opts(algo=Q.QS_ALGO_KERNELIZE, precision=precision, fuse_kmax=6,
                                                 mlp=net, shm_variant=2, shm_max_active=shm_max))]
            if contrast:
                plans.append(Q.Plan(n, g, Q.default_opts(algo=Q.QS_ALGO_KERNELIZE, precision=precision,
                                                         fuse_kmax=6, shm_variant=2, shm_max_active=shm_max)))
            for plan in plans:
                for k in range(plan.stats().num_kernels):
                    sub = g[plan.kernel_gates(k)]
                    if plan.kernel(k).type == Q.QS_KERNEL_FUSED:
                        opts = Q.default_opts(algo=Q.QS_ALGO_ORDERED, fuse_kmax=6, precision=precision, cost=fcost)
                    else:
                        opts = Q.default_opts(algo=Q.QS_ALGO_GREEDY, fuse_kmax=0, shm_max_active=14)
                    specs.append((sub, opts, opts.cost))
        Xn, yn, kinds = _time_specs(n, specs, reps, st, s, threads)
        Xn = np.asarray(Xn, dtype=np.float32)
        yn = np.asarray(yn, dtype=np.float32)
        # bias of the current model on the kernels its own plans chose
        pred = predict(net, Xn, stream=s)
        bias = float(np.mean(np.exp(pred - yn)))
        Xr, yr = np.concatenate([Xr, Xn]), np.concatenate([yr, yn])
        # held-out parts are split before the planner's choices are weighted
        rtr, rva, rte = split(len(yr), seed + 1)
        parts = [np.concatenate(p) for p in (
            [X[base[0]]] + [Xr[rtr]] * weight, [y[base[0]]] + [yr[rtr]] * weight,
            [X[base[1]], Xr[rva]], [y[base[1]], yr[rva]], [X[base[2]], Xr[rte]], [y[base[2]], yr[rte]])]
        if ensemble > 1:
            net, metrics = train_ensemble((parts[0], parts[1]), (parts[2], parts[3]), (parts[4], parts[5]),
                                          k=ensemble, seed=seed, tau=tau, epochs=epochs)
        else:
            net, metrics = train_parts((parts[0], parts[1]), (parts[2], parts[3]), (parts[4], parts[5]),
                                       epochs=epochs, seed=seed, tau=tau)
        history.append({"kernels": int(len(yn)), "fused": int(sum(kinds)), "pred_over_actual": bias})
        if log:
            log(f"refinement round {r + 1}: +{len(yn)} kernels ({sum(kinds)} fused), "
                f"predicted/actual on them before retraining {bias:.3f}, "
                f"test mean rel err {metrics['test']['mean_rel_err']:.3f}")
    rtr, rva, rte = split(len(yr), seed + 1)
    test_idx = np.concatenate([base[2], len(y) + rte]).astype(np.int64)
    metrics["refinement"] = history
    return net, np.concatenate([X, Xr]), np.concatenate([y, yr]), metrics, test_idx


def plan_gain(net, seeds=range(101, 110), n=26, gates=5000, shm_max=12, reps=3, stream=None, log=None,
              workload="mixed"):
    """The learned model's plan-level gain: for each seed, the mixed circuit
    (5000 gates) planned by Kernelize with the analytic table and with the
    learned cost under the same options (|A| <= shm_max, fused 3xTF32
    kernels allowed), each plan timed on a resident n-qubit state (the
    median of `reps` runs after one warm-up).  Returns per-seed circuit
    times and kernel counts and the gain sum(analytic) / sum(learned)."""
    import torch
    from synth import circuits as C
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    buf = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    st = Q.State(n, buf.data_ptr())
    out = {"n": n, "workload": workload, "shm_max_active": shm_max, "seeds": [], "analytic_ms": [], "learned_ms": [],
           "analytic_kernels": [], "learned_kernels": [], "learned_fused": []}

    def timed(plan):
        st.set_zero(s)
        st.run(plan, s)
        timer = Q.Timer(plan, reps)
        for _ in range(reps):
            st.run_timed(plan, timer, s)
        ms, runs = timer.read()
        return float(np.sum(ms)) / runs

    for seed in seeds:
        g = C.mixed_circuit(n, gates, seed) if workload == "mixed" else C.entangling_circuit(n, 40, seed)
        base = dict(algo=Q.QS_ALGO_KERNELIZE, precision=Q.QS_PREC_TF32X3, fuse_kmax=6, shm_max_active=shm_max)
        pa = Q.Plan(n, g, Q.default_opts(**base))
        pl = Q.Plan(n, g, Q.default_opts(mlp=net, **base))
        out["seeds"].append(int(seed))
        out["analytic_ms"].append(timed(pa))
        out["learned_ms"].append(timed(pl))
        out["analytic_kernels"].append(int(pa.stats().num_kernels))
        out["learned_kernels"].append(int(pl.stats().num_kernels))
        out["learned_fused"].append(int(pl.stats().num_fused))
        if log:
            log(f"seed {seed}: analytic {out['analytic_ms'][-1]:.2f} ms ({out['analytic_kernels'][-1]} kernels), "
                f"learned {out['learned_ms'][-1]:.2f} ms ({out['learned_kernels'][-1]} kernels, "
                f"{out['learned_fused'][-1]} fused)")
    out["gain"] = float(np.sum(out["analytic_ms"]) / np.sum(out["learned_ms"]))
    return out


def _unpack(theta, F, H):
    o = 0
    out = {}
    for name, shape in (("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H,)), ("b3", (1,))):
        size = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + size], dtype=np.float64).reshape(shape)
        o += size
    return out


def merge_ensemble(nets):
    """One network whose output is the mean of the given networks' outputs
    (same features F and width H each): their first layers side by side
    (F x kH), the second weight matrix block-diagonal (ReLU acts element by
    element, so the blocks never mix), the output weights divided by k and
    the output biases averaged."""
    F, H, k = nets[0].features, nets[0].hidden, len(nets)
    ps = [_unpack(n.get_params(), F, H) for n in nets]
    W1 = np.concatenate([p["W1"] for p in ps], axis=1)
    b1 = np.concatenate([p["b1"] for p in ps])
    W2 = np.zeros((k * H, k * H))
    for i, p in enumerate(ps):
        W2[i * H:(i + 1) * H, i * H:(i + 1) * H] = p["W2"]
    b2 = np.concatenate([p["b2"] for p in ps])
    W3 = np.concatenate([p["W3"] for p in ps]) / k
    b3 = np.array([np.mean([p["b3"][0] for p in ps])])
    net = Q.Mlp(F, k * H)
    net.set_params(np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3, b3]).astype(np.float32))
    return net


def train_ensemble(train_set, val_set, test_set, k=4, seed=0, tau=0.5, **kw):
    """k networks (seeds seed..seed+k-1) on the same parts, merged into one
    whose prediction is their mean; metrics of the merged network."""
    import torch
    nets = [train_parts(train_set, val_set, test_set, seed=seed + i, tau=tau, **kw)[0] for i in range(k)]
    net = merge_ensemble(nets)
    s = torch.cuda.current_stream().cuda_stream
    metrics = {name: evaluate(net, part[0], part[1], stream=s, tau=tau) for name, part in
               (("train", train_set), ("validation", val_set), ("test", test_set))}
    metrics["ensemble"] = k
    return net, metrics


def split(count, seed=0, fractions=(0.8, 0.1, 0.1)):
    perm = np.random.default_rng(seed).permutation(count)
    a = int(fractions[0] * count)
    b = a + int(fractions[1] * count)
    return perm[:a], perm[a:b], perm[b:]


def train(X, y, hidden=128, epochs=200, batch=256, lr=1e-3, seed=0, stream=None, log=None, tau=0.5):
    """Trains a fresh network on (X, y) with an 80/10/10 split; returns the
    network and a metrics dict (MSE of ln time; mean |relative error| of
    time) for the train, validation and test parts."""
    tr, va, te = split(len(y), seed)
    return train_parts((X[tr], y[tr]), (X[va], y[va]), (X[te], y[te]), hidden, epochs, batch, lr, seed,
                       stream, log, tau)


def train_parts(train_set, val_set, test_set, hidden=128, epochs=200, batch=256, lr=1e-3, seed=0,
                stream=None, log=None, tau=0.5):
    """Trains on train_set with the expectile-tau loss of ln(time) (tau =
    0.5: mean squared error; larger: pessimistic), keeps the epoch with the
    best validation loss, reports metrics on all three (X, y) parts."""
    import torch
    Xtr, ytr = train_set
    dev = torch.device("cuda")
    Xd = torch.from_numpy(np.ascontiguousarray(Xtr, dtype=np.float32)).to(dev)
    yd = torch.from_numpy(np.ascontiguousarray(ytr, dtype=np.float32)).to(dev)
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    net = Q.Mlp(Xtr.shape[1], hidden, seed)
    net.set_expectile(tau)
    # centre the output on the mean target so training starts close
    theta = net.get_params()
    theta[-1] = float(np.mean(ytr))
    net.set_params(theta)
    rng = np.random.default_rng(seed + 1)
    best, best_theta = float("inf"), net.get_params()
    for ep in range(epochs):
        order = rng.permutation(len(ytr))
        for b0 in range(0, len(order), batch):
            idx = torch.from_numpy(order[b0:b0 + batch]).to(dev)
            xb = Xd.index_select(0, idx).contiguous()
            tb = yd.index_select(0, idx).contiguous()
            net.train_step(xb.data_ptr(), tb.data_ptr(), len(idx), lr, s)
        if ep % 10 == 9 or ep == epochs - 1:
            v = evaluate(net, val_set[0], val_set[1], stream=s, tau=tau)["loss"]
            if v < best:
                best, best_theta = v, net.get_params()
            if log:
                log(f"epoch {ep + 1}: validation MSE {v:.4f}")
    net.set_params(best_theta)
    metrics = {name: evaluate(net, part[0], part[1], stream=s, tau=tau) for name, part in
               (("train", train_set), ("validation", val_set), ("test", test_set))}
    return net, metrics


def predict(net, X, bf16=True, stream=None) -> np.ndarray:
    import torch
    dev = torch.device("cuda")
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
    out = torch.empty(len(X), dtype=torch.float32, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    net.forward(Xd.data_ptr(), len(X), out.data_ptr(), bf16, s)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def evaluate(net, X, y, bf16=True, stream=None, tau=0.5) -> dict:
    """MSE and expectile-tau loss of ln(time), mean and median |relative
    error| of time, and the mean predicted/actual time ratio."""
    if len(y) == 0:
        return {"mse": float("nan"), "loss": float("nan"), "mean_rel_err": float("nan")}
    p = predict(net, X, bf16, stream)
    d = p - y
    rel = np.abs(np.exp(d) - 1.0)
    w = np.where(d < 0, 2 * tau, 2 * (1 - tau))
    return {"mse": float(np.mean(d ** 2)), "loss": float(np.mean(w * d ** 2)),
            "mean_rel_err": float(np.mean(rel)), "median_rel_err": float(np.median(rel)),
            "pred_over_actual": float(np.mean(np.exp(d)))}


def save(net, path=MODEL_PATH, meta=None) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, theta=net.get_params(), features=net.features, hidden=net.hidden,
             meta=json.dumps(meta or {}))


def load(path=MODEL_PATH):
    d = np.load(path)
    net = Q.Mlp(int(d["features"]), int(d["hidden"]))
    net.set_params(d["theta"])
    return net, json.loads(str(d["meta"]))


def main(argv=None):
    """python -m paper_2408_09055_gb300.costmodel [--count N] [--out PATH]:
    times `count` kernels on a 30-qubit state, trains, saves the model and the
    dataset beside it.  With --evaluate it loads the model at --out instead
    and prints plan_gain's JSON for the given qubits, seeds and workload."""
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=6144)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--out", default=MODEL_PATH)
    ap.add_argument("--refine-rounds", type=int, default=6)
    ap.add_argument("--data", default=None, help="reuse timed kernels saved by an earlier run")
    ap.add_argument("--tau", type=float, default=0.5,
                    help="expectile of ln(time) the network learns (0.5: mean squared error)")
    ap.add_argument("--ensemble", type=int, default=1, help="networks averaged into the saved one")
    ap.add_argument("--contrast", action="store_true",
                    help="refinement also times the analytic plans' kernels of the same circuits")
    ap.add_argument("--evaluate", action="store_true",
                    help="load the model at --out and time analytic against learned plans (plan_gain)")
    ap.add_argument("--qubits", type=int, default=30, help="state size for --evaluate")
    ap.add_argument("--seeds", default="100-109", help="circuit seeds for --evaluate, e.g. 100-109")
    ap.add_argument("--workload", default="mixed", choices=("mixed", "entangling"))
    a = ap.parse_args(argv)
    if a.evaluate:
        lo, _, hi = a.seeds.partition("-")
        net, _ = load(a.out)
        r = plan_gain(net, seeds=range(int(lo), int(hi or lo) + 1), n=a.qubits, log=print, workload=a.workload)
        print(json.dumps(r))
        return
    if a.data:
        d = np.load(a.data)
        X, y, meta = d["X"], d["y"], json.loads(str(d["meta"]))
    else:
        X, y, meta = generate(count=a.count, seed=a.seed)
    if a.ensemble > 1:
        tr, va, te = split(len(y), a.seed)
        net, metrics = train_ensemble((X[tr], y[tr]), (X[va], y[va]), (X[te], y[te]), k=a.ensemble, seed=a.seed,
                                      tau=a.tau, epochs=a.epochs)
    else:
        net, metrics = train(X, y, epochs=a.epochs, seed=a.seed, log=print, tau=a.tau)
    test_idx = split(len(y), a.seed)[2]
    if a.refine_rounds:
        net, X, y, metrics, test_idx = refine(net, X, y, rounds=a.refine_rounds, seed=a.seed, epochs=a.epochs,
                                              tau=a.tau, ensemble=a.ensemble, contrast=a.contrast)
        meta["refine_rounds"] = a.refine_rounds
        meta["count"] = int(len(y))
    np.savez(os.path.splitext(a.out)[0] + "_data.npz", X=X, y=y, test_idx=test_idx, meta=json.dumps(meta))
    meta["metrics"] = metrics
    meta["tau"] = a.tau
    meta["ensemble"] = a.ensemble
    meta["contrast"] = bool(a.contrast)
    save(net, a.out, meta)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
