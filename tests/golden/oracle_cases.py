"""Small seeded cases run through the FP64 oracle, for the change-control
fixture `oracle_small.json` beside this file.

The fixture holds the cases' inputs and the oracle's outputs on them.  It is
written by `make_oracle_golden.py` and read back by
`tests/test_oracle_golden.py`, both through `run()` below, which calls only
`oracle/`.  Its outputs are not pins of correctness (the pins live in the
`test_oracle_*.py` files and check the oracle against finite differences,
closed forms, brute force and independent implementations); they make any
change to the oracle's arithmetic visible: a commit that changes the oracle's
results has to rewrite the fixture and name the passage of the paper, or the
reading of it, that the change follows.

The cases use non-unit physics (mass 2.5, kT 2.49, LJ sigma 1.1 and epsilon
0.7, dt 0.004, gamma 0.5), a mixed torsion + distance CV set and a residual
ensemble, so that every scaling of the step enters some output."""
import numpy as np

SYS_SCALARS = ("n_beads", "n_cv", "seed", "mass", "kT", "dt", "gamma", "bond_k", "bond_r0", "angle_k",
               "angle_theta0", "lj_eps", "lj_sigma", "lj_rc", "output_freq")


def encode(o):
    """numpy arrays and scalars to JSON-ready values (floats keep their repr)."""
    if isinstance(o, dict):
        return {k: encode(v) for k, v in o.items()}
    if isinstance(o, (list, tuple)):
        return [encode(v) for v in o]
    if isinstance(o, np.ndarray):
        return {"dtype": str(o.dtype), "shape": list(o.shape), "data": o.ravel().tolist()}
    if isinstance(o, np.generic):
        return o.item()
    return o


def decode(o):
    if isinstance(o, dict) and set(o) == {"dtype", "shape", "data"}:
        return np.array(o["data"], dtype=o["dtype"]).reshape(o["shape"])
    if isinstance(o, dict):
        return {k: decode(v) for k, v in o.items()}
    if isinstance(o, list):
        return [decode(v) for v in o]
    return o


def system_from(d):
    from paper_2408_14070_gb300 import inputs as I
    sp = I.SystemParams(**{k: d[k] for k in SYS_SCALARS})
    sp.dihedral_k = np.asarray(d["dihedral_k"], dtype=np.float64)
    sp.dihedral_delta = np.asarray(d["dihedral_delta"], dtype=np.float64)
    sp.cv_atoms = np.asarray(d["cv_atoms"], dtype=np.int32)
    return sp


def ensemble_from(d):
    from paper_2408_14070_gb300 import inputs as I
    return I.EnsembleParams(d["n_models"], d["n_in"], d["n_layers"], d["width"], bool(d["resnet"]),
                            np.asarray(d["weights"], dtype=np.float32), d["trust_lo"], d["trust_hi"])


def run(inp):
    """The oracle's outputs on the decoded inputs `inp`."""
    import oracle
    from oracle import mcmc as orc_mcmc
    from oracle import select as orc_select
    from oracle import train as orc_train
    sp = system_from(inp["system"])
    ens = ensemble_from(inp["ensemble"])
    x0 = inp["x0"]
    dist = sp.cv_atoms[:, 2] < 0
    out = {}
    out["philox"] = oracle.philox(inp["philox_counters"], inp["philox_seed"])
    for w in range(x0.shape[0]):
        U, f, terms = oracle.ff(sp, x0[w].astype(np.float64))
        s, J = oracle.cvs(sp, x0[w].astype(np.float64))
        e = oracle.ensemble(ens, s, sp.cv_atoms)
        t = oracle.total(sp, x0[w], ens)
        r = oracle.total(sp, x0[w], mode=2, s0=inp["s0"][w], kappa=inp["kappa"][w])
        out[f"walker{w}"] = {"U_ff": U, "f_ff": f, "terms": terms, "s": s, "J": J,
                             "Fs": e["Fs"], "eps": e["eps"], "Abar": e["Abar"], "sigma": e["sigma"],
                             "gradA": e["gradA"], "f_biased": t["f"], "f_restrained": r["f"],
                             "U_restraint": r["U_restraint"]}
    ex = oracle.explore(sp, x0, inp["explore_steps"], ens=ens, energy=True, n_threads=1)
    out["explore"] = {k: ex[k] for k in ("cv", "eps", "energy", "x", "v")}
    lb = oracle.label(sp, x0, inp["s0"], inp["kappa"], inp["label_steps"], inp["label_equil"],
                      inp["label_blocks"], n_threads=1)
    out["label"] = {k: lb[k] for k in ("mf", "se", "std", "x", "v")}
    tr = inp["train"]
    w_out, losses, _, _ = orc_train.train(ens.weights, ens.n_in, ens.n_layers, ens.width, ens.resnet,
                                          tr["s"], tr["mf"], tr["idx"], init_lr=tr["init_lr"],
                                          decay_rate=tr["decay_rate"], decay_steps=tr["decay_steps"],
                                          dropout_rate=tr["dropout_rate"], dropout_seed=tr["dropout_seed"],
                                          dist=dist)
    out["train"] = {"weights": w_out, "losses": losses}
    sl = inp["select"]
    res = orc_select.select(sl["cv"], sl["eps"], sl["trust_lo"], sl["trust_hi"], sl["threshold"], sl["lower"],
                            sl["upper"], True, sl["max_selection"], w=sl["weights"], periodic=~dist)
    out["select"] = {"selected": np.asarray(res["selected"], dtype=np.int64), "n_clusters": res["n_clusters"],
                     "threshold": res["threshold"]}
    mc = inp["mcmc"]
    m = orc_mcmc.run(ens.weights, sp.n_cv, ens.n_layers, ens.width, ens.resnet, mc["s0"], mc["n_steps"],
                     mc["n_burn"], mc["kT"], mc["step_size"], mc["seed"], mc["bins"], (0, 1), dist=dist,
                     lo=mc["lo"], hi=mc["hi"])
    out["mcmc"] = {"s": m["s"], "n_accepted": m["n_accepted"], "hist1": m["hist1"], "hist2": m["hist2"]}
    return out
