"""Learned fusion cost model: training data, training, planner evaluation.

The model (an MLP in libqudit, see include/qudit.h "learned cost model")
predicts the device time of one launch from its 12 launch features.  Training
data are timings the simulator itself produces: random single gates and
random fused blocks (up to 3 qudits, D <= 64) applied to large registers
(>= 1e8 amplitudes), each launch timed with CUDA events through a plan with an
explicit segmentation.  Everything here is orchestration over the C ABI; the
timing, training and inference work runs in the library's kernels.
"""
from __future__ import annotations

import math
import os
import time
from typing import Iterable, Sequence

import numpy as np

from . import qudit as L
from . import workloads as wl
from .workloads import Gate

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "cost_model_gb300.npz")

# Registers the training launches run on (complex64, 1.3e8 .. 2.7e8 amplitudes).
TRAIN_REGISTERS = (
    [3] * 17,                      # 1.29e8
    [2] * 8 + [4] * 10,            # 2.68e8
    [3] * 11 + [2] * 6 + [4] * 2,  # 1.81e8
    [4] * 6 + [3] * 6 + [2] * 6,   # 1.91e8
    [2] * 27,                      # 1.34e8
)


# Registers above 2^31 amplitudes (64-bit index kernels; 34-50 GB complex64).
LARGE_REGISTERS = (
    [3] * 18 + [2] * 4,  # 6.2e9
    [2] * 8 + [4] * 12,  # 4.3e9
)


def register_size(dims: Sequence[int]) -> int:
    return int(np.prod([int(d) for d in dims]))


def random_diag_run(rng: np.random.Generator, dims: Sequence[int]):
    """2-10 diagonal gates (phases on one qudit, controlled phases, two-qudit
    phase tables) spread over a contiguous range of 4-12 qudits whose table
    has at most 2^22 entries: one diagonal-run launch."""
    n = len(dims)
    for _ in range(50):
        width = int(rng.integers(4, min(12, n) + 1))
        lo = int(rng.integers(0, n - width + 1))
        if int(np.prod(dims[lo:lo + width])) <= (1 << 22):
            break
    else:
        lo, width = 0, 4
    qs = list(range(lo, lo + width))
    out = []
    for _ in range(int(rng.integers(2, 11))):
        r = rng.random()
        if r < 0.3:
            q = int(rng.choice(qs))
            out.append(Gate("Z", (q,), param=int(rng.integers(1, dims[q]))))
        elif r < 0.7:
            c, t = (int(x) for x in rng.choice(qs, size=2, replace=False))
            out.append(Gate("DIAG", (t,), (c,), (int(rng.integers(0, dims[c])),),
                            matrix=np.exp(2j * np.pi * rng.random(dims[t]))))
        else:
            a, b = (int(x) for x in rng.choice(qs, size=2, replace=False))
            out.append(Gate("DIAG", (a, b), matrix=np.exp(2j * np.pi * rng.random(dims[a] * dims[b]))))
    # make the run span more than three qudits (beyond the block limit)
    used = {q for g in out for q in tuple(g.targets) + tuple(g.controls or ())}
    for q in qs:
        if len(used) > 3:
            break
        if q not in used:
            out.append(Gate("Z", (q,), param=1))
            used.add(q)
    return out


def random_dense_with_run(rng: np.random.Generator, dims: Sequence[int]):
    """A dense gate on one or two qudits (at most 16 states) followed by a
    diagonal run over 4-12 qudits: one dense launch with a table epilogue."""
    n = len(dims)
    for _ in range(50):
        k = int(rng.integers(1, 3))
        qs = [int(x) for x in rng.choice(n, size=k, replace=False)]
        if int(np.prod([dims[q] for q in qs])) <= 16:
            break
    else:
        qs = [0]
    D = int(np.prod([dims[q] for q in qs]))
    return [Gate("U", tuple(qs), matrix=wl.haar_unitary(D, rng))] + random_diag_run(rng, dims)


def random_launch(rng: np.random.Generator, dims: Sequence[int], dmax: int = 64):
    """Gates that form one launch: a single permutation/diagonal gate, a
    single dense gate, a fused block of two dense gates over 2-3 qudits, a
    fused block of 2-4 permutations with phases over 2-3 qudits, a run of
    diagonal gates over 4-12 qudits, or a dense gate followed by such a run."""
    n = len(dims)
    kind = rng.choice(["mono", "dense", "block", "block", "block", "monoblock", "diagrun", "denserun"])
    if kind == "diagrun":
        return random_diag_run(rng, dims)
    if kind == "denserun":
        return random_dense_with_run(rng, dims)
    if kind == "monoblock":
        # fused permutations with phases (shifts, clocks, controlled shifts)
        # on 2-3 qudits: the product runs on the mono kernel
        for _ in range(50):
            k = int(rng.integers(2, 4))
            qs = [int(x) for x in rng.choice(n, size=k, replace=False)]
            if int(np.prod([dims[q] for q in qs])) <= 32:
                break
        else:
            qs = [0, 1]
        out = []
        for _ in range(int(rng.integers(2, 5))):
            t = int(rng.choice(qs))
            others = [q for q in qs if q != t]
            sub = rng.integers(0, 3)
            if sub == 0:
                out.append(Gate("X", (t,), param=int(rng.integers(1, dims[t]))))
            elif sub == 1:
                out.append(Gate("Z", (t,), param=1))
            else:
                c = int(rng.choice(others))
                out.append(Gate("X", (t,), (c,), (int(rng.integers(0, dims[c])),), int(rng.integers(1, dims[t]))))
        if len({q for g in out for q in (tuple(g.targets) + tuple(g.controls or ()))}) < 2:
            c = [q for q in qs if q != out[0].targets[0]][0]
            out.append(Gate("Z", (c,), param=1))
        return out
    if kind == "mono":
        q = int(rng.integers(0, n))
        sub = rng.integers(0, 3)
        if sub == 0:
            return [Gate("X", (q,), param=int(rng.integers(1, dims[q])))]
        if sub == 1:
            return [Gate("Z", (q,), param=1)]
        c = int(rng.choice([x for x in range(n) if x != q]))
        return [Gate("X", (q,), (c,), (int(rng.integers(0, dims[c])),), int(rng.integers(1, dims[q])))]
    if kind == "dense":
        k = int(rng.integers(1, 3))
        for _ in range(20):
            qs = [int(x) for x in rng.choice(n, size=k, replace=False)]
            D = int(np.prod([dims[q] for q in qs]))
            if D <= 32:
                break
        ctrl = ()
        lv = None
        if rng.random() < 0.3:
            c = int(rng.choice([x for x in range(n) if x not in qs]))
            ctrl, lv = (c,), (int(rng.integers(0, dims[c])),)
        return [Gate("U", tuple(qs), ctrl, lv, matrix=wl.haar_unitary(D, rng))]
    for _ in range(50):
        k = int(rng.integers(2, 4))
        qs = [int(x) for x in rng.choice(n, size=k, replace=False)]
        D = int(np.prod([dims[q] for q in qs]))
        if D <= dmax:
            break
    else:
        qs = [0, 1]
    if len(qs) == 2:
        return [Gate("U", (qs[0],), matrix=wl.haar_unitary(dims[qs[0]], rng)),
                Gate("U", (qs[1],), matrix=wl.haar_unitary(dims[qs[1]], rng))]
    a, b, c = qs
    return [Gate("U", (a, b), matrix=wl.haar_unitary(dims[a] * dims[b], rng)),
            Gate("U", (b, c), matrix=wl.haar_unitary(dims[b] * dims[c], rng))]


def time_launch(reg: int, gates, reps: int = 3, kind: int = -1) -> float:
    """Median device time (ms) of the single launch the gates form (in the
    given kernel form; -1: the analytic cost model's choice)."""
    ga = L.GateArray(gates)
    plan = L.qd_plan_create_segmented(reg, ga, [(0, len(gates) - 1)], [kind])
    try:
        L.qd_plan_profile(plan, True)
        ts = []
        for _ in range(reps):
            L.qd_plan_run(plan)
            ms, _, _ = L.qd_plan_timings(plan)
            ts.append(float(ms.sum()))
        return float(np.median(ts))
    finally:
        L.qd_plan_destroy(plan)


def generate(n_samples: int, seed: int = 0, registers: Iterable[Sequence[int]] = TRAIN_REGISTERS,
             precision: int = L.QD_C64, reps: int = 3, stream: int = 0, log=None):
    """Features X[n, 12] and targets y[n] = log(launch time in microseconds)."""
    rng = np.random.default_rng(seed)
    regs = [list(r) for r in registers]
    X, y = [], []
    per = int(math.ceil(n_samples / len(regs)))
    t0 = time.time()
    for dims in regs:
        h = L.qd_create(dims, None, precision, 0, 0, stream)
        try:
            for i in range(per):
                if len(y) >= n_samples:
                    break
                gates = random_launch(rng, dims, 64 if precision == L.QD_C64 else 32)
                # every feasible form of the launch is timed (both block
                # kernels for 9 <= D <= 32, a block or a dense part + run),
                # each sample with the features of the form that ran
                ga = L.GateArray(gates)
                for kind, f in L.qd_segment_forms(h, ga, 0, len(gates) - 1):
                    ms = time_launch(h, gates, reps, kind)
                    X.append(f)
                    y.append(math.log(max(ms, 1e-4) * 1e3))
        finally:
            L.qd_destroy(h)
        if log:
            log(f"register {dims}: {len(y)} samples, {time.time() - t0:.1f} s")
    return np.array(X, np.float32), np.array(y, np.float32)


def train(X, y, epochs: int = 80, batch: int = 256, lr: float = 2e-3, seed: int = 0):
    """Train a new model on the GPU; returns (model handle, final loss)."""
    m = L.qd_model_create()
    loss = L.qd_model_train(m, X, y, epochs, batch, lr, seed)
    return m, loss


def kernel_source_sha() -> str:
    """Hash of the library's CUDA and host sources: the kernels a set of
    training timings was taken on."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(HERE, "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(f.encode())
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def save(model: int, path: str = DEFAULT_WEIGHTS, **meta) -> None:
    w = L.qd_model_get(model)
    np.savez(path, **w, **{k: np.asarray(v) for k, v in meta.items()})


def load(path: str = DEFAULT_WEIGHTS) -> int:
    d = np.load(path)
    m = L.qd_model_create()
    L.qd_model_set(m, d["params"], d["feat_mean"], d["feat_std"], float(d["y_mean"]), float(d["y_std"]))
    return m


# ---------------------------------------------------------------------------
# Planner evaluation
# ---------------------------------------------------------------------------

def eval_circuit(seed: int, n_active: int = 10, ngates: int = 40, spectators: Sequence[int] = (),
                  dim_choices=(2, 3, 4)):
    """A random circuit on n_active qudits (dims from dim_choices) placed
    among spectator qudits (which no gate touches), so that the register is
    large while the circuit is small enough for exhaustive planning."""
    rng = np.random.default_rng(seed)
    active = [int(x) for x in rng.choice(dim_choices, size=n_active)]
    dims = list(spectators[: len(spectators) // 2]) + active + list(spectators[len(spectators) // 2:])
    off = len(spectators) // 2
    sub = wl.random_circuit(active, ngates, seed, wl.C0_MIX + ("U2",))
    gates = []
    for g in sub:
        gates.append(Gate(g.kind, tuple(t + off for t in g.targets), tuple(c + off for c in g.controls),
                          g.levels, g.param, g.matrix))
    return dims, gates


def plan_time(reg: int, gates, plan_kind=None, segments=None, reps: int = 3) -> float:
    """Median device time (ms) of a whole plan (graph replay)."""
    ga = L.GateArray(gates)
    plan = (L.qd_plan_create_segmented(reg, ga, segments) if segments is not None
            else L.qd_plan_create(reg, ga, plan_kind))
    try:
        L.qd_plan_profile(plan, True)
        ts = []
        for _ in range(reps):
            L.qd_plan_run(plan)
            ms, _, _ = L.qd_plan_timings(plan)
            ts.append(float(ms.sum()))
        return float(np.median(ts))
    finally:
        L.qd_plan_destroy(plan)


def _is_diag(g) -> bool:
    return g.kind in ("Z", "DIAG")


def _dense_then_run(gates, dims, a, b, kmax):
    """Gates a..b as a dense part (<= kmax qudits, <= 16 states) followed by a
    nonempty run of diagonal gates whose covering range has <= 2^24 states."""
    k = b
    while k >= a and _is_diag(gates[k]):
        k -= 1
    if k < a or k == b:
        return False
    pre = set()
    for g in gates[a:k + 1]:
        pre |= set(g.controls or ()) | set(g.targets)
    run = set()
    for g in gates[k + 1:b + 1]:
        run |= set(g.controls or ()) | set(g.targets)
    return (len(pre) <= kmax and int(np.prod([dims[q] for q in pre])) <= 16
            and int(np.prod(dims[min(run):max(run) + 1])) <= (1 << 24))


def exhaustive_measured(reg: int, dims: Sequence[int], gates, kmax: int = 3, dmax: int = 64, reps: int = 3,
                        record=None):
    """The measured optimum: the minimum-time contiguous segmentation, where every
    candidate segment's cost is its measured launch time (dynamic program
    over prefixes; a segment of several gates must span <= kmax qudits of
    total dimension <= dmax, be a run of diagonal gates whose covering qudit
    range gives a table of <= 2^24 entries, or a dense part followed by such a
    run; every feasible kernel form of a segment is timed -- a dense block of
    9 <= D <= 32 on the CUDA cores and on the tensor cores, a block or a
    dense part + run -- and the fastest counts).  record: a list that
    receives (features, ms) of every timed form.  Returns (segments, summed
    measured ms)."""
    n = len(gates)
    cost = {}
    best = [0.0] + [math.inf] * n
    back = [-1] * (n + 1)
    for i in range(1, n + 1):
        qs = set()
        all_diag = True
        for j in range(i - 1, -1, -1):
            qs |= set(gates[j].controls or ()) | set(gates[j].targets)
            all_diag = all_diag and _is_diag(gates[j])
            in_block = len(qs) <= kmax and int(np.prod([dims[q] for q in qs])) <= dmax
            in_run = all_diag and int(np.prod(dims[min(qs):max(qs) + 1])) <= (1 << 24)
            in_dt = _dense_then_run(gates, dims, j, i - 1, kmax)
            if j < i - 1 and not (in_block or in_run or in_dt):
                break  # unions only grow as j decreases
            seg = (j, i - 1)
            if seg not in cost:
                ts = []
                sub = L.GateArray(gates[j:i])
                for kind, f in L.qd_segment_forms(reg, sub, 0, i - j - 1):
                    ts.append(time_launch(reg, gates[j:i], reps, kind))
                    if record is not None:
                        record.append((f, ts[-1]))
                cost[seg] = min(ts)
            c = best[j] + cost[seg]
            if c < best[i]:
                best[i], back[i] = c, j
    segs, i = [], n
    while i > 0:
        segs.append((back[i], i - 1))
        i = back[i]
    return segs[::-1], best[n]


# Spectator sets of the training circuits (the evaluation circuits use
# (3, 3, 3, 3, 3, 2, 2, 2, 2) and seeds from 7000).
TRAIN_SPECTATORS = (
    (3, 3, 3, 3, 3, 2, 2, 2, 2),
    (2,) * 12,
    (3,) * 8,
    (4, 4, 4, 4, 4, 4),
    (2, 2, 2, 2, 3, 3, 3, 3, 3, 3),
    (3, 3, 2, 2, 2, 2, 2, 2, 2, 2, 2),
)


def large_spectators(seed: int, cap: int = 1 << 33):
    """Spectator ququarts that put the circuit of this seed on a register of
    2^31..2^33 amplitudes (64-bit index kernels; <= 68.7 GB complex64)."""
    dims, _ = eval_circuit(seed)
    k = int(math.floor(math.log(cap / register_size(dims), 4)))
    return (4,) * max(k, 0)


def circuit_samples(n_circuits: int, seed: int = 20000, reps: int = 3, log=None, large: bool = False):
    """Training samples from the planner's own queries: every candidate
    segment of random circuits (the shape of the evaluation circuits, other
    seeds, varied spectators; large: spectators up to 2^31..2^33
    amplitudes), each feasible form timed.  Returns X, y."""
    rng = np.random.default_rng(seed)
    X, y = [], []
    t0 = time.time()
    for c in range(n_circuits):
        spect = (large_spectators(seed + c) if large
                 else TRAIN_SPECTATORS[int(rng.integers(len(TRAIN_SPECTATORS)))])
        dims, gates = eval_circuit(seed + c, spectators=spect)
        h = L.qd_create(dims, None, L.QD_C64, 0, 0, 0)
        try:
            rec = []
            exhaustive_measured(h, dims, gates, reps=reps, record=rec)
            for f, ms in rec:
                X.append(f)
                y.append(math.log(max(ms, 1e-4) * 1e3))
        finally:
            L.qd_destroy(h)
        if log and ((c + 1) % 10 == 0 or large):
            log(f"circuits {c + 1}/{n_circuits}: {len(y)} samples, {time.time() - t0:.1f} s")
    return np.array(X, np.float32), np.array(y, np.float32)


def evaluate(model: int, n_circuits: int = 4, seed: int = 7000, spectators=(3, 3, 3, 3, 3, 2, 2, 2, 2),
             measured: bool = True, reps: int = 3, log=None):
    """Measured plan times (ms) on evaluation circuits: one gate per launch, the
    greedy and exhaustive plans under the analytic cost model, the learned
    plan, and (measured=True) the exhaustive optimum over measured segment costs."""
    rows = []
    for c in range(n_circuits):
        dims, gates = eval_circuit(seed + c, spectators=spectators)
        h = L.qd_create(dims, None, L.QD_C64, 0, 0, 0)
        try:
            L.qd_set_cost_model(h, model)
            row = {"N": register_size(dims), "gates": len(gates),
                   "per_gate": plan_time(h, gates, L.QD_PLAN_NONE, reps=reps),
                   "greedy": plan_time(h, gates, L.QD_PLAN_GREEDY, reps=reps),
                   "exhaustive_analytic": plan_time(h, gates, L.QD_PLAN_EXHAUSTIVE, reps=reps),
                   "learned": plan_time(h, gates, L.QD_PLAN_LEARNED, reps=reps)}
            if measured:
                segs, opt = exhaustive_measured(h, dims, gates, reps=reps)
                row["measured_optimum"] = opt
            rows.append(row)
            if log:
                log(str(row))
        finally:
            L.qd_destroy(h)
    return rows


def main(argv=None):
    import argparse
    import json

    ap = argparse.ArgumentParser(description="generate timings, train the cost model, evaluate the planners")
    ap.add_argument("--samples", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=80)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--circuits", type=int, default=4)
    ap.add_argument("--no-measured-optimum", action="store_true",
                    help="skip the exhaustive search over measured segment costs (slow)")
    ap.add_argument("--large-samples", type=int, default=0,
                    help="extra samples on registers above 2^31 amplitudes (64-bit index kernels)")
    ap.add_argument("--circuit-samples", type=int, default=0,
                    help="training circuits whose candidate segments are all timed (the planner's own queries)")
    ap.add_argument("--large-circuit-samples", type=int, default=0,
                    help="training circuits as --circuit-samples on registers of 2^31..2^33 amplitudes")
    ap.add_argument("--base-data", default=None,
                    help="npz (X, y) of earlier samples to train on together with the new ones")
    args = ap.parse_args(argv)
    from .build import build
    build()
    L.load()
    log = lambda m: print(m, flush=True)  # noqa: E731
    t0 = time.time()
    parts_X, parts_y = [], []
    if args.base_data:
        d = np.load(args.base_data)
        parts_X.append(d["X"])
        parts_y.append(d["y"])
        log(f"base data: {len(d['y'])} samples")
    if args.samples > 0:
        X, y = generate(args.samples, args.seed, log=log)
        parts_X.append(X)
        parts_y.append(y)
    if args.large_samples > 0:
        X, y = generate(args.large_samples, args.seed + 1, registers=LARGE_REGISTERS, reps=2, log=log)
        parts_X.append(X)
        parts_y.append(y)
    if args.circuit_samples > 0:
        X, y = circuit_samples(args.circuit_samples, 20000 + args.seed, log=log)
        parts_X.append(X)
        parts_y.append(y)
    if args.large_circuit_samples > 0:
        X, y = circuit_samples(args.large_circuit_samples, 30000 + args.seed, reps=2, log=log, large=True)
        parts_X.append(X)
        parts_y.append(y)
    X, y = np.concatenate(parts_X), np.concatenate(parts_y)
    gen_s = time.time() - t0
    n = len(y)
    idx = np.random.default_rng(args.seed).permutation(n)
    tr, te = idx[: int(0.9 * n)], idx[int(0.9 * n):]
    m, loss = train(X[tr], y[tr], args.epochs, seed=args.seed)
    pred = L.qd_model_predict(m, X[te])
    resid = pred - y[te]
    r2 = 1.0 - float(np.sum(resid ** 2) / np.sum((y[te] - y[te].mean()) ** 2))
    save(m, args.out, samples=n, train_loss=loss, test_r2=r2, test_rmse_log=float(np.sqrt(np.mean(resid ** 2))),
         source_sha=kernel_source_sha(), seed=args.seed)
    np.savez(os.path.splitext(args.out)[0] + "_data.npz", X=X, y=y)
    rows = evaluate(m, args.circuits, measured=not args.no_measured_optimum, log=log)
    tot = {k: float(sum(r[k] for r in rows)) for k in rows[0] if k not in ("N", "gates")}
    print(json.dumps({"samples": n, "gen_s": gen_s, "train_loss": loss, "test_r2": r2,
                      "source_sha": kernel_source_sha(),
                      "test_rmse_log": float(np.sqrt(np.mean(resid ** 2))), "plan_ms_totals": tot,
                      "circuits": rows}), flush=True)
    L.qd_model_destroy(m)


if __name__ == "__main__":
    main()
