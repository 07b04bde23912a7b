"""Train the format-selector network on timings of the exhaustive search.

    python -m paper_1004_3719_gb300.train_selector --train 2000 --test 200 \
        --weights paper_1004_3719_gb300/selector_weights.npy --report <file.md>

1. Corpus: the generated family of matrices (10^4-2*10^6 rows; banded,
   block-diagonal, uniform and power-law structure; +-1 share 0-100%;
   moduli 3, 65521, 2^31-1), made by worker processes (spawn) while the GPU
   works.  For every matrix: the device features, then the exhaustive search
   (every valid format of every non-empty bin timed on a row sample).
2. Training samples are the (matrix, bin) pairs: input = 16 matrix features +
   6 bin features; target = log(t_format / t_best) for each valid format and
   log(t_pm / t_nopm) for the +-1 flag.  The network is trained on the GPU by
   the library's own forward / loss / backward / Adam kernels.
3. Evaluation on the held-out matrices: the cost of a choice is the sum over
   bins of (sample time per entry) x (entries of the bin); the report gives
   exhaustive-best cost / chosen cost ("% of exhaustive-best throughput") for
   the network, the heuristic table and a single fixed CSR width, and a few
   whole-matrix timings of the resulting plans.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NUM_BINS, NUM_FORMATS = 17, 10


def _make(args):
    import gen
    seed, index, rows_lo, rows_hi = args
    A = gen.selector_matrix(seed, index, rows_lo=rows_lo, rows_hi=rows_hi)
    return index, A


def samples_of(feat, binfeat, tune, min_sample_nnz=256):
    """Training rows of one matrix: (x[k][22], target[k][11], mask[k][11], bins)."""
    X, T, Mk, bins = [], [], [], []
    t = tune["times"].astype(np.float64)
    pm = tune["pm_times"].astype(np.float64)
    for b in range(1, NUM_BINS):
        if tune["sample_nnz"][b] < min_sample_nnz or not np.any(np.isfinite(t[b])):
            continue
        tb = t[b]
        ok = np.isfinite(tb) & (tb > 0)
        best = tb[ok].min()
        target = np.zeros(NUM_FORMATS + 1)
        mask = np.zeros(NUM_FORMATS + 1)
        target[:NUM_FORMATS][ok] = np.log(tb[ok] / best)
        mask[:NUM_FORMATS][ok] = 1.0
        if np.isfinite(pm[b, 1]) and pm[b, 0] > 0 and pm[b, 1] > 0:
            target[NUM_FORMATS] = np.log(pm[b, 1] / pm[b, 0])
            mask[NUM_FORMATS] = 1.0
        X.append(np.concatenate([feat, binfeat[b]]))
        T.append(target)
        Mk.append(mask)
        bins.append(b)
    return X, T, Mk, bins


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
    if data is None:
        jobs = [(args.seed, i, args.rows_lo, args.rows_hi) for i in range(n_all)]
        for k, (i, A) in enumerate(pool.imap(_make, jobs, chunksize=1)):
            feat, binfeat = sel.matrix_features(A)
            tune = sel.tune_bins(A)
            heur = sel.heuristic_choose(A)
            recs.append(dict(index=i, name=A.name, nrows=A.nrows, nnz=A.nnz, feat=feat,
                             binfeat=binfeat, tune=tune, heur=heur, fixed=fixed_csr_choice(A),
                             nnz_b=bin_nnz(A)))
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
    rows = []
    for r in test_recs:
        best_c = best_cost(r["tune"], r["nnz_b"])
        learned = learned_choice(net, r)
        rows.append(dict(name=r["name"], nrows=r["nrows"], nnz=r["nnz"],
                         learned=best_c / choice_cost(r["tune"], r["nnz_b"], learned),
                         heuristic=best_c / choice_cost(r["tune"], r["nnz_b"], r["heur"]),
                         fixed_csr=best_c / choice_cost(r["tune"], r["nnz_b"], r["fixed"])))
    summ = {k: dict(mean=float(np.mean([x[k] for x in rows])), median=float(np.median([x[k] for x in rows])),
                    min=float(np.min([x[k] for x in rows])))
            for k in ("learned", "heuristic", "fixed_csr")}
    e2e = end_to_end(ff, sel, test_recs[:args.e2e], args) if args.e2e > 0 else []
    result = dict(train_matrices=len(train_recs), test_matrices=len(test_recs),
                  train_samples=int(Xtr.shape[0]), corpus_seconds=round(t_corpus, 1),
                  train_seconds=round(t_train, 1), losses=losses, summary=summ, e2e=e2e)
    print(json.dumps(result))
    if args.report:
        write_report(args, result, rows)


def learned_choice(net, r):
    """The network's choice for a corpus record (same rule as the library's
    inference: argmin over valid formats, +-1 when the predicted log ratio < 0)."""
    import torch
    X = np.array([np.concatenate([r["feat"], r["binfeat"][b]]) for b in range(NUM_BINS)],
                 dtype=np.float32)
    out, _ = net.forward(torch.from_numpy(X).to(net.dev))
    out = out.cpu().numpy()
    t = r["tune"]["times"]
    best = np.zeros((NUM_BINS, 3), dtype=np.int32)
    for b in range(1, NUM_BINS):
        valid = np.isfinite(t[b])
        if not valid.any():
            continue
        scores = np.where(valid, out[b, :NUM_FORMATS], np.inf)
        best[b] = [int(np.argmin(scores)), int(out[b, NUM_FORMATS] < 0), 1]
    return best


def end_to_end(ff, sel, recs, args):
    """Whole-matrix y = A x timings (L2 flushed between calls) of the plans
    from the network, the exhaustive search, the heuristic table and the
    plain fixed-width CSR format."""
    import torch

    import gen
    out = []
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    sink = torch.zeros(64 << 20, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    for r in recs:
        A = gen.selector_matrix(args.seed, r["index"], rows_lo=args.rows_lo, rows_hi=args.rows_hi)
        x = torch.from_numpy(gen.uniform_block(7, A.ncols, 1, A.modulus).view(np.int32)).cuda()
        y = torch.empty(A.nrows, dtype=torch.int32, device="cuda")
        res = {"name": A.name, "nnz": A.nnz}
        plans = {"learned": sel.create_binned(A, sel.selector_choose(A), transpose_mode=2),
                 "exhaustive": sel.create_binned(A, r["tune"]["best"], transpose_mode=2),
                 "heuristic": sel.create_binned(A, r["heur"], transpose_mode=2),
                 "fixed_csr": ff.Matrix.from_csr(A, priority_format=ff.FMT.CSR, transpose_mode=2)}
        for k, M in plans.items():
            for _ in range(3):
                ff.spmv_apply(M.handle, x, 1, y, 1, 1, 1, 0, st.cuda_stream)
            ts = []
            for _ in range(10):
                flush.fill_(1)
                s_ = sink.sum()  # noqa: F841
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                ff.spmv_apply(M.handle, x, 1, y, 1, 1, 1, 0, st.cuda_stream)
                e1.record(st)
                ts.append((e0, e1))
            torch.cuda.synchronize()
            res[k + "_us"] = round(1e3 * float(np.median([a.elapsed_time(b) for a, b in ts])), 1)
        out.append(res)
    return out


def write_report(args, result, rows):
    s = result["summary"]
    lines = [
        "# Format selector: training and held-out evaluation",
        "",
        f"Command: `python -m paper_1004_3719_gb300.train_selector --train {args.train} --test {args.test} "
        f"--seed {args.seed} --steps {args.steps}` (one GB300).",
        "",
        f"* corpus: {result['train_matrices']} training + {result['test_matrices']} held-out matrices, "
        f"{result['train_samples']} (matrix, bin) training samples; corpus {result['corpus_seconds']} s, "
        f"training {result['train_seconds']} s",
        f"* loss (masked squared error of log time ratios): {result['losses'][0][1]:.4f} at step 1, "
        f"{result['losses'][-1][1]:.4f} at step {result['losses'][-1][0]}",
        "",
        "Held-out share of exhaustive-best throughput (cost model: per-bin sample times x bin entries):",
        "",
        "| chooser | mean | median | min |",
        "|---|---|---|---|",
    ]
    for k in ("learned", "heuristic", "fixed_csr"):
        lines.append(f"| {k} | {100 * s[k]['mean']:.1f}% | {100 * s[k]['median']:.1f}% | {100 * s[k]['min']:.1f}% |")
    if result["e2e"]:
        lines += ["", "Whole-matrix y = A x (µs, median of 10, L2 flushed):", "",
                  "| matrix | nnz | learned | exhaustive | heuristic | fixed CSR |", "|---|---|---|---|---|---|"]
        for e in result["e2e"]:
            lines.append(f"| {e['name']} | {e['nnz']} | {e['learned_us']} | {e['exhaustive_us']} | "
                         f"{e['heuristic_us']} | {e['fixed_csr_us']} |")
    with open(args.report, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
