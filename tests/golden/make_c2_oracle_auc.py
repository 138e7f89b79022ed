"""Writes tests/golden/c2_oracle_auc.txt: the FP64 sequential oracle's
link-prediction AUCs on the full-size workload (R-MAT scale 20, edge factor
16, 80/20 split; d = 128, k = 3, lr 0.01, e = 400 epochs of |E| updates,
p = 0.3, Alg. 4 coarsening and Alg. 2 with copy projection), seeds 1-3.

Calls only oracle/ and synth/ (about 30 minutes of one core per seed; the
seeds run in parallel processes):
    python tests/golden/make_c2_oracle_auc.py
"""
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_oracle_auc.txt")
C2 = dict(d=128, k=3, lr=0.01, e=400, p=0.3)


def one_seed(seed):
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    sp = synth.workload("rmat20")
    gr = sp.train
    t0 = time.time()
    M, info = oracle.embed(gr.rowptr, gr.col, seed=seed, epoch_unit="E", **C2)
    fp, fn = synth.fit_pairs(gr)
    return (seed, oracle.link_auc(M, fp, fn), oracle.link_auc(M, sp.test_pos, sp.test_neg), info["epochs"],
            time.time() - t0)


def main():
    ctx = mp.get_context("spawn")
    with ctx.Pool(3) as pool:
        rows = pool.map(one_seed, [1, 2, 3])
    with open(OUT, "w") as f:
        f.write("# FP64 sequential oracle on R-MAT scale 20 (ef 16, 80/20 split), d=128, k=3, lr=0.01,\n"
                "# e=400 epochs of |E| updates, p=0.3, copy projection; passes per level %s.\n"
                "# training-edge AUC: synth.fit_pairs(train) (400000 sampled edges u<v vs as many uniform\n"
                "# pairs, seed 5); held-out AUC: the split's test edges vs its negatives.\n"
                "# Written by tests/golden/make_c2_oracle_auc.py (oracle/ and synth/ only).\n"
                "# columns: seed  training_edge_auc  heldout_auc\n" % (rows[0][3],))
        for seed, fit, held, _, dt in rows:
            f.write("%d %.6f %.6f\n" % (seed, fit, held))
    for r in rows:
        print(r)


if __name__ == "__main__":
    main()
