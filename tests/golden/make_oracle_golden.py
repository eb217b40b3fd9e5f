"""Writes oracle_small.json: the inputs of a few small seeded cases and the
FP64 oracle's outputs on them (see oracle_cases.py for what the fixture is
for).  Calls only the seeded input generators and oracle/.

    python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, HERE)

import oracle_cases as G  # noqa: E402


def make_inputs():
    import oracle
    from paper_2408_14070_gb300 import inputs as I
    sp = I.make_system(14, 3, 3, n_dist=1, dist_span=5, mass=2.5, kT=2.49, lj_sigma=1.1, lj_eps=0.7,
                       dt=0.004, gamma=0.5, output_freq=5)
    x0 = I.make_chains(2, sp, 3)
    ens = I.make_ensemble(3, 6, 2, 8, 3, resnet=True)
    # trust levels around the walkers' model deviations, so that the switch
    # takes a value strictly between 0 and 1 for at least one of them
    e = [oracle.ensemble(ens, oracle.cvs(sp, x0[w].astype(np.float64))[0], sp.cv_atoms)["eps"] for w in range(2)]
    ens.trust_lo, ens.trust_hi = 0.5 * min(e), 1.5 * max(e)
    rng = np.random.default_rng(2024)
    s_now = np.array([oracle.cvs(sp, x0[w].astype(np.float64))[0] for w in range(2)])
    s0 = s_now + rng.uniform(-0.3, 0.3, size=s_now.shape)
    kappa = rng.uniform(50.0, 300.0, size=s_now.shape)
    dist = I.cv_is_distance(sp)
    s_train = rng.uniform(-np.pi, np.pi, size=(16, 3))
    s_train[:, dist] = rng.uniform(2.0, 5.0, size=(16, int(dist.sum())))
    train = {"s": s_train, "mf": rng.normal(0.0, 1.0, size=(16, 3)),
             "idx": rng.integers(0, 16, size=(3, 3, 4)), "init_lr": 1e-2, "decay_rate": 0.9,
             "decay_steps": 2, "dropout_rate": 0.1, "dropout_seed": 7}
    cv_sel = rng.uniform(-np.pi, np.pi, size=(120, 3))
    cv_sel[:, dist] = rng.uniform(2.0, 5.0, size=(120, int(dist.sum())))
    select = {"cv": cv_sel, "eps": rng.uniform(0.0, 2.0, size=120), "trust_lo": 0.3, "trust_hi": 1.6,
              "threshold": 0.5, "lower": 6, "upper": 9, "max_selection": 5,
              "weights": np.array([1.0, 2.0, 0.5])}
    s_mc = rng.uniform(-np.pi, np.pi, size=(8, 3))
    s_mc[:, dist] = rng.uniform(2.5, 4.5, size=(8, int(dist.sum())))
    lo = np.where(dist, 2.0, 0.0)
    hi = np.where(dist, 5.0, 0.0)
    mcmc = {"s0": s_mc, "n_steps": 60, "n_burn": 10, "kT": 2.49, "step_size": 0.3, "seed": 11, "bins": 8,
            "lo": lo, "hi": hi}
    sysd = {k: getattr(sp, k) for k in G.SYS_SCALARS}
    sysd.update(dihedral_k=sp.dihedral_k, dihedral_delta=sp.dihedral_delta, cv_atoms=sp.cv_atoms)
    ensd = {"n_models": ens.n_models, "n_in": ens.n_in, "n_layers": ens.n_layers, "width": ens.width,
            "resnet": int(ens.resnet), "weights": ens.weights, "trust_lo": ens.trust_lo, "trust_hi": ens.trust_hi}
    ctr = np.array([[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4], [7, 0, 9, 0x80000000]], dtype=np.uint32)
    return {"system": sysd, "ensemble": ensd, "x0": x0, "s0": s0, "kappa": kappa,
            "philox_counters": ctr, "philox_seed": 0x0123456789ABCDEF,
            "explore_steps": 20, "label_steps": 120, "label_equil": 20, "label_blocks": 4,
            "train": train, "select": select, "mcmc": mcmc}


def main():
    import oracle
    oracle.build()
    inp = G.decode(json.loads(json.dumps(G.encode(make_inputs()))))
    out = G.run(inp)
    doc = {"about": "inputs of small seeded cases and the FP64 oracle's outputs on them; written by "
                    "make_oracle_golden.py, read by test_oracle_golden.py",
           "inputs": G.encode(inp), "outputs": G.encode(out)}
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(doc, f, indent=None, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    main()
