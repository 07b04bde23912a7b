"""Train the format-selector network on timings of the exhaustive search.

    python -m paper_1004_3719_gb300.train_selector --train 2000 --test 200 \
        --weights paper_1004_3719_gb300/selector_weights.npy --report <file.md>

1. Corpus: the generated family of matrices (10^4-2*10^6 rows; banded,
   block-diagonal, uniform and power-law structure; +-1 share 0-100%;
   moduli 3, 65521, 2^31-1), made by worker processes (spawn) while the GPU
   works.  For every matrix: the device features, then the exhaustive search
   (every valid format of every non-empty bin timed on a row sample).
2. Whole-plan timings of every matrix: y = A x with the binned plan of the
   heuristic table (t_H), the binned plan of the exhaustive search's table
   (t_E) and the x-panel plan (t_P), L2 flushed before each call.
3. Training samples are the (matrix, bin) pairs: input = 16 matrix features +
   6 bin features; target = log(t_format / t_best) for each valid format and
   log(t_pm / t_nopm) for the +-1 flag; and one matrix-level sample per
   matrix: the 16 features with every bin feature set to MATRIX_INPUT,
   target = log(t_P / t_H) and log(t_E / t_H).  The network is trained on the
   GPU by the library's own forward / loss / backward / Adam kernels.
4. Evaluation on the held-out matrices: (a) per bin, the cost of a choice is
   the sum over bins of (sample time per entry) x (entries of the bin); the
   report gives exhaustive-best cost / chosen cost ("% of exhaustive-best
   throughput") for the network, the heuristic table and a single fixed CSR
   width; (b) whole plan, the best of t_H, t_E, t_P over the time of the
   layout each chooser picks; (c) whole-matrix timings of the handles that
   FMT.AUTO builds under each selector.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import re
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1004_3719_gb300._lib import (LAYOUT_BINNED, LAYOUT_NETBINS, LAYOUT_PANEL,  # noqa: E402
                                       LAYOUT_PANEL_Q1, LAYOUT_PANEL_Q2, LAYOUT_PANEL_Q4,
                                       MATRIX_INPUT, MLP_OUT, NUM_BIN_FEATURES, NUM_BINS,
                                       NUM_FORMATS, OUT_NETBINS, OUT_PANEL, OUT_PM,
                                       SEL_NET_MARGIN, SEL_Q_MARGIN, SEL_VERIFY_MARGIN)

# whole-plan timing keys: binned with the heuristic table (H) and with the
# exhaustive table (E), x-panel with clusters of 1, 2 and 4 CTAs (P1, P2, P4)
LAYOUT_KEY = {LAYOUT_BINNED: "H", LAYOUT_NETBINS: "E", LAYOUT_PANEL_Q1: "P1",
              LAYOUT_PANEL_Q2: "P2", LAYOUT_PANEL_Q4: "P4", LAYOUT_PANEL: "P"}


def _make(args):
    import gen
    seed, index, rows_lo, rows_hi = args
    A = gen.selector_matrix(seed, index, rows_lo=rows_lo, rows_hi=rows_hi)
    return index, A


def samples_of(feat, binfeat, tune, min_sample_nnz=256):
    """Training rows of one matrix's bins: (x[k][22], target[k][13], mask[k][13], bins)."""
    X, T, Mk, bins = [], [], [], []
    t = tune["times"].astype(np.float64)
    pm = tune["pm_times"].astype(np.float64)
    for b in range(1, NUM_BINS):
        if tune["sample_nnz"][b] < min_sample_nnz or not np.any(np.isfinite(t[b])):
            continue
        tb = t[b]
        ok = np.isfinite(tb) & (tb > 0)
        best = tb[ok].min()
        target = np.zeros(MLP_OUT)
        mask = np.zeros(MLP_OUT)
        target[:NUM_FORMATS][ok] = np.log(tb[ok] / best)
        mask[:NUM_FORMATS][ok] = 1.0
        if np.isfinite(pm[b, 1]) and pm[b, 0] > 0 and pm[b, 1] > 0:
            target[OUT_PM] = np.log(pm[b, 1] / pm[b, 0])
            mask[OUT_PM] = 1.0
        X.append(np.concatenate([feat, binfeat[b]]))
        T.append(target)
        Mk.append(mask)
        bins.append(b)
    return X, T, Mk, bins


def matrix_sample(feat, plan_us):
    """The matrix-level training row: (x[22], target[13], mask[13]), or None
    when the heuristic binned plan was not timed."""
    tH = plan_us.get("H", np.nan)
    if not (np.isfinite(tH) and tH > 0):
        return None
    x = np.concatenate([feat, np.full(NUM_BIN_FEATURES, MATRIX_INPUT)])
    target = np.zeros(MLP_OUT)
    mask = np.zeros(MLP_OUT)
    outs = [(OUT_NETBINS, "E")] + [(OUT_PANEL + i, f"P{q}") for i, q in enumerate((1, 2, 4))]
    for k, t in ((k, plan_us.get(key, np.nan)) for k, key in outs):
        if np.isfinite(t) and t > 0:
            target[k] = np.log(t / tH)
            mask[k] = 1.0
    return x, target, mask


def panel_rule(A):
    """The layout FMT.AUTO takes under the heuristic selector (the rule of
    panel_preferred in csrc/api.cu): x-panel when nnz >= 2^21 and nnz >=
    3 ncols."""
    return A.nnz >= (1 << 21) and A.nnz >= 3 * A.ncols


def time_handle(ff, M, x, y, flush, reps=7):
    """Median microseconds of one y = A x on handle M, L2 flushed before each
    call (3 untimed calls first)."""
    import torch
    st = torch.cuda.current_stream()
    for _ in range(3):
        ff.spmv_apply(M.handle, x, 1, y, 1, 1, 1, 0, st.cuda_stream)
    ts = []
    for _ in range(reps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ff.spmv_apply(M.handle, x, 1, y, 1, 1, 1, 0, st.cuda_stream)
        e1.record(st)
        ts.append((e0, e1))
    torch.cuda.synchronize()
    return 1e3 * float(np.median([a.elapsed_time(b) for a, b in ts]))


def whole_plan_times(ff, sel, A, tune, heur, flush):
    """Whole-plan microseconds of one matrix (NaN: not buildable): H, E,
    P1, P2, P4, and P = the x-panel plan with the builder's own cluster size
    ("q" holds that size)."""
    import torch
    x = torch.zeros(max(A.ncols, 1), dtype=torch.int32, device="cuda")
    y = torch.empty(max(A.nrows, 1), dtype=torch.int32, device="cuda")
    out = {}
    makers = {"H": lambda: sel.create_binned(A, heur, transpose_mode=2),
              "E": lambda: sel.create_binned(A, tune["best"], transpose_mode=2),
              "P": lambda: ff.Matrix.from_csr(A, priority_format=ff.FMT.PANEL, transpose_mode=2)}
    for q in (1, 2, 4):
        makers[f"P{q}"] = (lambda q=q: ff.Matrix.from_csr(A, priority_format=ff.FMT.PANEL, panel_cluster=q,
                                                          transpose_mode=2))
    out["q"] = 0
    for k, make in makers.items():
        if k.startswith("P") and k != "P" and k == f"P{out['q']}":
            out[k] = out["P"]  # the builder's own choice, timed already
            continue
        try:
            M = make()
        except ff.FFSPMVError:
            out[k] = np.nan
            continue
        d = M.describe()
        if k.startswith("P") and "panels" not in d:
            out[k] = np.nan
        else:
            out[k] = time_handle(ff, M, x, y, flush)
            if k == "P":
                mq = re.search(r"x (\d+) column groups", d)
                out["q"] = int(mq.group(1)) if mq else 0
        M.close()
    return out


def layout_time(plan_us, layout):
    t = plan_us.get(LAYOUT_KEY[layout], np.nan)
    return t if np.isfinite(t) else plan_us["H"]


def choice_cost(tune, nnz_b, best):
    """Sum over bins of (time per sampled entry) x (bin entries) for a choice
    best[17][3]; bins whose chosen format was not timed count at their worst
    timed format."""
    t = tune["times"].astype(np.float64)
    pm = tune["pm_times"].astype(np.float64)
    total = 0.0
    for b in range(1, NUM_BINS):
        sn = tune["sample_nnz"][b]
        if sn <= 0 or not np.any(np.isfinite(t[b])):
            continue
        f = int(best[b][0])
        tb = t[b][f] if np.isfinite(t[b][f]) else np.nanmax(t[b])
        if best[b][1] and np.isfinite(pm[b, 1]) and pm[b, 0] > 0:
            tb *= pm[b, 1] / pm[b, 0]
        total += tb / sn * nnz_b[b]
    return total


def best_cost(tune, nnz_b):
    t = tune["times"].astype(np.float64)
    pm = tune["pm_times"].astype(np.float64)
    total = 0.0
    for b in range(1, NUM_BINS):
        sn = tune["sample_nnz"][b]
        if sn <= 0 or not np.any(np.isfinite(t[b])):
            continue
        tb = np.nanmin(t[b])
        if np.isfinite(pm[b, 1]):
            tb = min(tb, tb * pm[b, 1] / pm[b, 0])
        total += tb / sn * nnz_b[b]
    return total


def fixed_csr_choice(A):
    """One CSR lane width for every bin: the power of two nearest below the
    mean row length (the plain single-launch CSR's rule)."""
    L = np.diff(A.row_ptr)
    ne = max(1, int((L > 0).sum()))
    mean = A.nnz / ne
    g = 1
    while g * 2 <= mean and g < 32:
        g *= 2
    f = 1 + int(np.log2(g))
    best = np.zeros((NUM_BINS, 3), dtype=np.int32)
    best[1:, 0] = f
    best[1:, 2] = 1
    return best


def bin_nnz(A):
    """Entries per row-length bin of the binned layout."""
    L = np.diff(A.row_ptr)
    b = np.zeros(L.shape, dtype=np.int64)
    pos = L > 0
    b[pos] = np.minimum(16, 1 + np.ceil(np.log2(L[pos])).astype(np.int64))
    return np.bincount(b, weights=L, minlength=NUM_BINS)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--seed", type=int, default=1005)
    ap.add_argument("--rows-lo", type=int, default=10_000)
    ap.add_argument("--rows-hi", type=int, default=2_000_000)
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 4) - 2))
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--weights", default=os.path.join(HERE, "selector_weights.npy"))
    ap.add_argument("--corpus", default="", help="npz cache of the corpus (read if present)")
    ap.add_argument("--report", default="")
    ap.add_argument("--e2e", type=int, default=6, help="held-out matrices timed end to end")
    ap.add_argument("--matrix-weight", type=int, default=4,
                    help="copies of each matrix-level sample in the training set")
    args = ap.parse_args()

    ctx = mp.get_context("spawn")
    pool = ctx.Pool(args.workers)  # before the first GPU call
    import torch

    import paper_1004_3719_gb300 as ff
    from paper_1004_3719_gb300 import selector as sel
    ff.build()
    torch.cuda.set_device(0)
    n_all = args.train + args.test
    data = None
    if args.corpus and os.path.exists(args.corpus):
        data = dict(np.load(args.corpus, allow_pickle=True))
    t0 = time.time()
    recs = []
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    if data is None:
        jobs = [(args.seed, i, args.rows_lo, args.rows_hi) for i in range(n_all)]
        for k, (i, A) in enumerate(pool.imap(_make, jobs, chunksize=1)):
            feat, binfeat = sel.matrix_features(A)
            tune = sel.tune_bins(A)
            heur = sel.heuristic_choose(A)
            recs.append(dict(index=i, name=A.name, nrows=A.nrows, nnz=A.nnz, feat=feat,
                             binfeat=binfeat, tune=tune, heur=heur, fixed=fixed_csr_choice(A),
                             nnz_b=bin_nnz(A), plan_us=whole_plan_times(ff, sel, A, tune, heur, flush),
                             panel_rule=panel_rule(A)))
            if (k + 1) % 50 == 0:
                print(f"[corpus] {k + 1}/{n_all} matrices, {time.time() - t0:.0f} s", flush=True)
        if args.corpus:
            np.savez_compressed(args.corpus, recs=np.array(recs, dtype=object))
    else:
        recs = list(data["recs"])
    pool.close()
    t_corpus = time.time() - t0
    train_recs = [r for r in recs if r["index"] < args.train]
    test_recs = [r for r in recs if r["index"] >= args.train]

    def stack(rs):
        X, T, Mk = [], [], []
        for r in rs:
            x, t, mk, _ = samples_of(r["feat"], r["binfeat"], r["tune"])
            X += x
            T += t
            Mk += mk
            ms = matrix_sample(r["feat"], r["plan_us"])
            if ms is not None:
                X += [ms[0]] * args.matrix_weight
                T += [ms[1]] * args.matrix_weight
                Mk += [ms[2]] * args.matrix_weight
        return (np.array(X, dtype=np.float32), np.array(T, dtype=np.float32),
                np.array(Mk, dtype=np.float32))

    Xtr, Ttr, Mtr = stack(train_recs)
    dev = torch.device("cuda", 0)
    xd, td, md = (torch.from_numpy(a).to(dev) for a in (Xtr, Ttr, Mtr))
    net = sel.MLP(seed=args.seed)
    g = torch.Generator(device="cpu").manual_seed(args.seed)
    losses = []
    t1 = time.time()
    for step in range(1, args.steps + 1):
        idx = torch.randint(0, xd.shape[0], (min(args.batch, xd.shape[0]),), generator=g).to(dev)
        loss, _ = net.loss_and_grad(xd[idx].contiguous(), td[idx].contiguous(), md[idx].contiguous())
        lr = args.lr * (0.5 * (1 + np.cos(np.pi * step / args.steps)))  # cosine decay
        net.adam(lr=float(lr))
        if step % 200 == 0 or step == 1:
            losses.append((step, float(loss.item())))
    torch.cuda.synchronize()
    t_train = time.time() - t1
    params = net.params()
    np.save(args.weights, params.astype(np.float32))
    sel.selector_load(params)

    # held-out evaluation
    rows, whole = [], []
    for r in test_recs:
        best_c = best_cost(r["tune"], r["nnz_b"])
        learned, layout, alt = learned_choice(net, r)
        rows.append(dict(name=r["name"], nrows=r["nrows"], nnz=r["nnz"],
                         learned=best_c / choice_cost(r["tune"], r["nnz_b"], learned),
                         heuristic=best_c / choice_cost(r["tune"], r["nnz_b"], r["heur"]),
                         fixed_csr=best_c / choice_cost(r["tune"], r["nnz_b"], r["fixed"])))
        pu = r["plan_us"]
        if np.isfinite(pu.get("H", np.nan)):
            tb = np.nanmin([pu.get(k, np.nan) for k in ("H", "E", "P", "P1", "P2", "P4")])
            t_heur = pu["P"] if r["panel_rule"] and np.isfinite(pu.get("P", np.nan)) else pu["H"]
            t_exh = np.nanmin([pu.get("E", np.nan), pu.get("P", np.nan), np.inf])
            t_learned = layout_time(pu, layout)
            if alt >= 0:   # the timed check between the two families
                t_learned = min(t_learned, layout_time(pu, alt))
            whole.append(dict(name=r["name"], layout=layout, learned=tb / t_learned,
                              heuristic=tb / t_heur, exhaustive=tb / (t_exh if np.isfinite(t_exh) else pu["H"]),
                              learned_us=t_learned, heuristic_us=t_heur, verified=alt >= 0))
    summ = {k: dict(mean=float(np.mean([x[k] for x in rows])), median=float(np.median([x[k] for x in rows])),
                    min=float(np.min([x[k] for x in rows])))
            for k in ("learned", "heuristic", "fixed_csr")}
    summ_whole = {k: dict(mean=float(np.mean([x[k] for x in whole])), median=float(np.median([x[k] for x in whole])),
                          min=float(np.min([x[k] for x in whole])))
                  for k in ("learned", "heuristic", "exhaustive")} if whole else {}
    layouts = {n: int(sum(1 for w in whole if w["layout"] == v))
               for n, v in (("binned", LAYOUT_BINNED), ("netbins", LAYOUT_NETBINS), ("panel_q1", LAYOUT_PANEL_Q1),
                            ("panel_q2", LAYOUT_PANEL_Q2), ("panel_q4", LAYOUT_PANEL_Q4), ("panel", LAYOUT_PANEL))}
    total_us = {k: float(sum(w[k + "_us"] for w in whole)) for k in ("learned", "heuristic")}
    total_us["verified"] = int(sum(1 for w in whole if w["verified"]))
    e2e = end_to_end(ff, sel, test_recs[:args.e2e], args) if args.e2e > 0 else []
    result = dict(train_matrices=len(train_recs), test_matrices=len(test_recs),
                  train_samples=int(Xtr.shape[0]), corpus_seconds=round(t_corpus, 1),
                  train_seconds=round(t_train, 1), losses=losses, summary=summ,
                  whole_plan=summ_whole, layouts=layouts, total_us=total_us, e2e=e2e)
    print(json.dumps(result))
    if args.report:
        write_report(args, result, rows)


def learned_choice(net, r):
    """The network's choice for a corpus record, by the library's inference
    rule: per bin the argmin over valid formats and +-1 when the predicted log
    ratio is negative; the layout of least predicted whole-plan time (the
    heuristic binned plan counting 0).  Returns (best[17][3], layout, alt)."""
    import torch
    X = [np.concatenate([r["feat"], r["binfeat"][b]]) for b in range(NUM_BINS)]
    X.append(np.concatenate([r["feat"], np.full(NUM_BIN_FEATURES, MATRIX_INPUT)]))
    out, _ = net.forward(torch.from_numpy(np.array(X, dtype=np.float32)).to(net.dev))
    out = out.cpu().numpy()
    t = r["tune"]["times"]
    best = np.zeros((NUM_BINS, 3), dtype=np.int32)
    for b in range(1, NUM_BINS):
        valid = np.isfinite(t[b])
        if not valid.any():
            continue
        scores = np.where(valid, out[b, :NUM_FORMATS], np.inf)
        best[b] = [int(np.argmin(scores)), int(out[b, OUT_PM] < 0), 1]
    return best, layout_rule(out[NUM_BINS])[0], layout_rule(out[NUM_BINS])[1]


def layout_rule(o):
    """The library's whole-plan rule on the matrix-level outputs o: the
    least predicted time between the x-panel family (a cluster size only when
    it beats the other two by SEL_Q_MARGIN, else the builder's) and the
    binned family (the network's own table only when it beats the heuristic
    table by SEL_NET_MARGIN).  Returns (layout, alt): alt is the other
    family's layout when the two are predicted within SEL_VERIFY_MARGIN (the
    library then times both and keeps the faster), else -1."""
    pq = [float(o[OUT_PANEL + i]) for i in range(3)]
    kq = int(np.argmin(pq))
    second = min(pq[i] for i in range(3) if i != kq)
    vp = pq[kq]
    lp = (LAYOUT_PANEL_Q1 + kq) if second - vp > SEL_Q_MARGIN else LAYOUT_PANEL
    net = float(o[OUT_NETBINS]) < -SEL_NET_MARGIN
    vb = float(o[OUT_NETBINS]) if net else 0.0
    lb = LAYOUT_NETBINS if net else LAYOUT_BINNED
    layout = lp if vp < vb else lb
    alt = (lb if vp < vb else lp) if abs(vp - vb) < SEL_VERIFY_MARGIN else -1
    return layout, alt


def end_to_end(ff, sel, recs, args):
    """Whole-matrix y = A x timings (L2 flushed between calls) of the handles
    FMT.AUTO builds under the learned, exhaustive and heuristic selectors,
    and of the plain fixed-width CSR format."""
    import torch

    import gen
    out = []
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for r in recs:
        A = gen.selector_matrix(args.seed, r["index"], rows_lo=args.rows_lo, rows_hi=args.rows_hi)
        x = torch.from_numpy(gen.uniform_block(7, A.ncols, 1, A.modulus).view(np.int32)).cuda()
        y = torch.empty(A.nrows, dtype=torch.int32, device="cuda")
        res = {"name": A.name, "nnz": A.nnz}
        makers = {"learned": lambda: ff.Matrix.from_csr(A, selector=ff.SEL.LEARNED, transpose_mode=2),
                  "exhaustive": lambda: ff.Matrix.from_csr(A, selector=ff.SEL.EXHAUSTIVE, transpose_mode=2),
                  "heuristic": lambda: ff.Matrix.from_csr(A, transpose_mode=2),
                  "fixed_csr": lambda: ff.Matrix.from_csr(A, priority_format=ff.FMT.CSR, transpose_mode=2)}
        for k, make in makers.items():
            M = make()
            res[k + "_us"] = round(time_handle(ff, M, x, y, flush, reps=10), 1)
            res[k + "_layout"] = "panel" if "panels" in M.describe() else "binned"
            M.close()
        out.append(res)
    return out


def write_report(args, result, rows):
    s = result["summary"]
    lines = [
        "# Format selector: training and held-out evaluation",
        "",
        f"Command: `python -m paper_1004_3719_gb300.train_selector --train {args.train} --test {args.test} "
        f"--seed {args.seed} --steps {args.steps} --matrix-weight {args.matrix_weight} --e2e {args.e2e}` "
        "(one GB300).",
        "",
        f"* corpus: {result['train_matrices']} training + {result['test_matrices']} held-out matrices, "
        f"{result['train_samples']} training samples ((matrix, bin) pairs and matrix-level rows); corpus "
        f"{result['corpus_seconds']} s, training {result['train_seconds']} s",
        f"* loss (masked squared error of log time ratios): {result['losses'][0][1]:.4f} at step 1, "
        f"{result['losses'][-1][1]:.4f} at step {result['losses'][-1][0]}",
    ]
    w = result["whole_plan"]
    if w:
        t = result["total_us"]
        lines += ["", "## Whole-matrix time of y = A x (the headline)", "",
                  f"Summed over the held-out matrices: **{t['learned']:.0f} µs with the learned selector vs "
                  f"{t['heuristic']:.0f} µs with the heuristic AUTO rule**. Per matrix, the best whole-plan time "
                  "(binned with the heuristic table, binned with the exhaustive table, x-panel with 1, 2 or 4 CTAs "
                  "per cluster) over the time of the layout each chooser gets (learned: the library's rule on the "
                  "network's matrix-level outputs, with its timed check of close calls; heuristic: the AUTO panel "
                  "rule; exhaustive: the faster of its binned plan and the x-panel plan), L2 flushed, median of 7:",
                  "", "| chooser | mean | median | min |", "|---|---|---|---|"]
        for k in ("learned", "heuristic", "exhaustive"):
            lines.append(f"| {k} | {100 * w[k]['mean']:.1f}% | {100 * w[k]['median']:.1f}% | "
                         f"{100 * w[k]['min']:.1f}% |")
        lines += ["", f"Layouts the network picked: {result['layouts']}; {t['verified']} close calls checked by "
                  "timing both families."]
    if result["e2e"]:
        lines += ["", "FMT.AUTO handles built by the library under each selector, timed whole (µs, median of 10, "
                  "L2 flushed; layout in brackets):", "",
                  "| matrix | nnz | learned | exhaustive | heuristic | fixed CSR |", "|---|---|---|---|---|---|"]
        for e in result["e2e"]:
            lines.append(f"| {e['name']} | {e['nnz']} | {e['learned_us']} ({e['learned_layout']}) | "
                         f"{e['exhaustive_us']} ({e['exhaustive_layout']}) | "
                         f"{e['heuristic_us']} ({e['heuristic_layout']}) | {e['fixed_csr_us']} |")
    lines += ["", "## Per-bin format choice (cost model of the exhaustive search's sample timings)", "",
              "Held-out share of exhaustive-best throughput, the cost of a choice being the sum over bins of "
              "(sample time per entry) x (entries of the bin):", "",
              "| chooser | mean | median | min |", "|---|---|---|---|"]
    for k in ("learned", "heuristic", "fixed_csr"):
        lines.append(f"| {k} | {100 * s[k]['mean']:.1f}% | {100 * s[k]['median']:.1f}% | {100 * s[k]['min']:.1f}% |")
    with open(args.report, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
