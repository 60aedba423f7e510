"""Collect selector timings on the GPU, train the network on the GPU, evaluate
regret on held-out graphs and write the weights the library loads.

    python -m paper_2603_11645_gb300.selector_train --train 2000 --heldout 200 \
        --data-dir paper_2603_11645_gb300/selector_data

Resumes from existing CSVs in --data-dir (timings are not re-collected).
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np

from . import selector as S


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--heldout", type=int, default=200)
    ap.add_argument("--data-dir", default=os.path.join(os.path.dirname(__file__), "selector_data"))
    ap.add_argument("--epochs", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=S.WEIGHTS_PATH)
    args = ap.parse_args()
    os.makedirs(args.data_dir, exist_ok=True)
    tr = os.path.join(args.data_dir, f"train_{args.train}.csv")
    ho = os.path.join(args.data_dir, f"heldout_{args.heldout}.csv")
    if not os.path.exists(tr):
        S.generate_dataset("train", args.train, tr, args.reps)
    if not os.path.exists(ho):
        S.generate_dataset("heldout", args.heldout, ho, args.reps)
    Xtr, Ttr, _ = S.load_dataset(tr)
    Xho, Tho, fam = S.load_dataset(ho)
    model = S.train(Xtr, Ttr, args.epochs, args.lr, args.seed)
    model["margin"] = S.fit_margin(model, Xtr, Ttr)
    pred = S.predict_host(model, Xho)
    sel = S.choose(pred, model["margin"])
    cc = np.ones(len(Tho), dtype=int)
    best = Tho.argmin(1)
    report = {
        "heldout_graphs": int(len(Tho)),
        "selector_regret": S.regret(Tho, sel),
        "always_cc_euler_regret": S.regret(Tho, cc),
        "always_bfs_regret": S.regret(Tho, np.zeros(len(Tho), dtype=int)),
        "oracle_choice_counts": {s: int((best == k).sum()) for k, s in enumerate(S.STRATS)},
        "selector_choice_counts": {s: int((sel == k).sum()) for k, s in enumerate(S.STRATS)},
        "selector_sum_ratio": float(Tho[np.arange(len(Tho)), sel].sum() / Tho.min(1).sum()),
        "margin": model["margin"],
        "train_loss_first": model["loss_first"], "train_loss_last": model["loss_last"],
    }
    model["heldout_report"] = report
    with open(args.out, "w") as fh:
        json.dump(model, fh)
    print(json.dumps(report, indent=1))


if __name__ == "__main__":
    main()
