"""One JSON configuration per run: the workload, the time axis, the solver and the outputs.

A configuration is a JSON object with four sections; every key is optional and takes the
default below, and an unknown key is an error (a typo must not pass silently):

    {"workload": {"kind": "small-box" | "two-layer" | "realistic" | "candidate",
                  "seed": int | null, "crop": int | null, "candidate": int, "directions": [0, 1, 2]},
     "time":     {"n_steps": int, "band": [f1, f2] | null},
     "solver":   {"tol": 1e-8, "max_iter": 10000, "precision": "fp64" | "fp32" | "fp16",
                  "inner_iters": 45, "inner_rtol": 0.0125, "guess_order": 4,
                  "outer_op": "auto" | "fp64" | "dword", "batch_outer": 0,
                  "coarse_weight": 0.0, "coarse_relres": 0.0, "proj_dim": 0, "proj_relres": 0.0,
                  "share_dirs": 0},
     "output":   {"waveforms": path | null, "summary": path | null}}

The workload kinds are the seeded synthetic models of ``synth.configs`` (the paper's models are
not published): a small two-layer box, the two-layer 100 x 100 x 50 m model, the three-layer
1.2 x 1.2 x 0.3 km model (optionally its lateral crop), and a candidate of the mixed-precision
ensemble; ``seed`` null keeps the workload's own seed.  The time step is the workload's own
(its input samples are made for it); ``band`` (the Rayleigh-fit band) defaults to the
workload's.  The solver section maps one to one
onto ``gsw_solver_opts`` (``solver_kwargs``).  ``run`` uploads the model, runs the analyses of
the listed input directions (one batch), and returns the receiver histories and a summary that
repeats the resolved configuration, so every output carries the configuration that made it.
"""
import copy
import json

DEFAULTS = {
    "workload": {"kind": "small-box", "seed": None, "crop": None, "candidate": 0, "directions": [0]},
    "time": {"n_steps": 20, "band": None},
    "solver": {"tol": 1e-8, "max_iter": 10000, "precision": "fp64", "inner_iters": 45, "inner_rtol": 0.0125,
               "guess_order": 4, "outer_op": "auto", "batch_outer": 0, "coarse_weight": 0.0,
               "coarse_relres": 0.0, "proj_dim": 0, "proj_relres": 0.0, "share_dirs": 0},
    "output": {"waveforms": None, "summary": None},
}
KINDS = ("small-box", "two-layer", "realistic", "candidate")
PRECISIONS = {"fp64": 0, "fp32": 1, "fp16": 2}
OUTER_OPS = {"auto": 0, "fp64": 1, "dword": 2}


def resolve(cfg):
    """The configuration with every default filled in; raises ValueError on an unknown section
    or key, or on a value of the wrong kind."""
    if isinstance(cfg, str):
        with open(cfg) as f:
            cfg = json.load(f)
    if not isinstance(cfg, dict):
        raise ValueError("a run configuration is a JSON object")
    out = copy.deepcopy(DEFAULTS)
    for sec, vals in cfg.items():
        if sec not in DEFAULTS:
            raise ValueError("unknown section %r (sections: %s)" % (sec, ", ".join(DEFAULTS)))
        if not isinstance(vals, dict):
            raise ValueError("section %r must be an object" % sec)
        for k, v in vals.items():
            if k not in DEFAULTS[sec]:
                raise ValueError("unknown key %s.%s" % (sec, k))
            out[sec][k] = v
    w, t, s = out["workload"], out["time"], out["solver"]
    if w["kind"] not in KINDS:
        raise ValueError("workload.kind must be one of %s" % (KINDS,))
    dirs = w["directions"]
    if not (isinstance(dirs, list) and dirs and all(d in (0, 1, 2) for d in dirs) and len(set(dirs)) == len(dirs)):
        raise ValueError("workload.directions must be a non-empty list of distinct values from 0, 1, 2")
    if not (isinstance(t["n_steps"], int) and t["n_steps"] > 0):
        raise ValueError("time.n_steps must be a positive integer")
    if t["band"] is not None and not (len(t["band"]) == 2 and 0.0 < t["band"][0] < t["band"][1]):
        raise ValueError("time.band must be [f1, f2] with 0 < f1 < f2")
    if s["precision"] not in PRECISIONS:
        raise ValueError("solver.precision must be one of %s" % (tuple(PRECISIONS),))
    if s["outer_op"] not in OUTER_OPS:
        raise ValueError("solver.outer_op must be one of %s" % (tuple(OUTER_OPS),))
    return out


def solver_kwargs(cfg):
    """Keyword arguments of ``Model.set_solver`` (the fields of gsw_solver_opts) from a
    resolved configuration."""
    s = cfg["solver"]
    return dict(tol=float(s["tol"]), max_iter=int(s["max_iter"]), precision=PRECISIONS[s["precision"]],
                inner_iters=int(s["inner_iters"]), inner_rtol=float(s["inner_rtol"]),
                guess_order=int(s["guess_order"]), outer_op=OUTER_OPS[s["outer_op"]],
                batch_outer=int(s["batch_outer"]), coarse_weight=float(s["coarse_weight"]),
                coarse_relres=float(s["coarse_relres"]), proj_dim=int(s["proj_dim"]),
                proj_relres=float(s["proj_relres"]), share_dirs=int(s["share_dirs"]))


def workload(cfg):
    """The seeded synthetic workload of a resolved configuration (``synth.configs``)."""
    from synth import configs

    w, n = cfg["workload"], cfg["time"]["n_steps"]
    d0 = w["directions"][0]
    seed = {} if w["seed"] is None else {"seed": int(w["seed"])}
    if w["kind"] == "small-box":
        return configs.small_box(n_steps=n, direction=d0, **seed)
    if w["kind"] == "two-layer":
        return configs.config1(n_steps=n, direction=d0)
    if w["kind"] == "realistic":
        return configs.config2(n_steps=n, crop=w["crop"], direction=d0, **seed)
    return configs.config4_candidate(int(w["candidate"]), n_steps=n, direction=d0)


def run(cfg, ctx=None):
    """Run the configured analyses on the GPU.  Returns (waveforms {direction: [n_rec, 3,
    n_steps]}, summary dict with the resolved configuration, the model's size, wall time and
    per-direction solver statistics); writes the outputs the configuration names."""
    import time

    import numpy as np

    from . import gsw

    cfg = resolve(cfg)
    wl = workload(cfg)
    own = ctx is None
    if own:
        ctx = gsw.Context(0)
    m = ctx.upload(wl["mesh"], wl["mat"], wl["rec_xy"])
    try:
        band = tuple(cfg["time"]["band"]) if cfg["time"]["band"] is not None else wl["band"]
        n = cfg["time"]["n_steps"]
        m.set_time(wl["dt"], n, band)
        for d in cfg["workload"]["directions"]:
            m.set_input(d, np.asarray(wl["p"][:n]))
        m.set_solver(**solver_kwargs(cfg))
        mask = sum(1 << d for d in cfg["workload"]["directions"])
        t0 = time.perf_counter()
        m.run(dirs_mask=mask)
        seconds = time.perf_counter() - t0
        waves = {d: m.waveforms(d) for d in cfg["workload"]["directions"]}
        summary = {"config": cfg, "workload": wl["name"], "dof": 3 * m.n_nodes, "dt": wl["dt"],
                   "seconds": seconds, "stats": {str(d): m.stats(d) for d in cfg["workload"]["directions"]}}
    finally:
        m.free()
        if own:
            ctx.close()
    out = cfg["output"]
    if out["waveforms"]:
        np.save(out["waveforms"], np.stack([waves[d] for d in cfg["workload"]["directions"]]))
    if out["summary"]:
        with open(out["summary"], "w") as f:
            json.dump(summary, f, indent=1)
    return waves, summary


if __name__ == "__main__":
    import sys

    if len(sys.argv) != 2:
        sys.exit("usage: python -m paper_2404_17754_gb300.runconfig CONFIG.json")
    _, summ = run(sys.argv[1])
    print(json.dumps(summ))
