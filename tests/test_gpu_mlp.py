"""Learned CG initial guess on the GPU against the CPU oracle of the MLP.

* tensor-core (BF16 operands, FP32 accumulation) inference vs the oracle's
  bf16-rounded forward pass;
* tensor-core training gradients (BF16 operands, FP32 accumulation) vs the
  oracle's gradient with the same rounding points, and vs its exact FP64
  backprop (pinned by finite differences);
* a run that trains on its first 500 steps and then applies the guess
  converges every step to the same 1e-8 relative residual and reproduces the
  plain run, and the trained network gains: a lower initial residual than the
  Newmark predictor and no more outer iterations;
* the data path (features, sampled nodes, targets, base guess, scales)
  against the oracle's.
"""
import numpy as np
import pytest

from oracle import mlp, newmark
from synth import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_17754_gb300 import build, gsw

    build.build()
    c = gsw.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def model(ctx):
    cfg = configs.small_box(n_steps=4)
    m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
    m.set_time(cfg["dt"], 4, cfg["band"])
    m.set_solver(tol=1e-8, precision=1)
    yield m
    m.free()


def _params(seed):
    rng = np.random.default_rng(seed)
    th = mlp.init(seed) + 0.05 * rng.standard_normal(mlp.N_PARAMS)
    return th.astype(np.float32).astype(np.float64)  # what the device holds


def test_tensor_core_inference_matches_oracle(model):
    th = _params(1)
    model.mlp_params(th)
    X = np.random.default_rng(2).standard_normal((1000, 16)).astype(np.float32)  # partial last tile
    out = model.mlp_forward(X)
    ref = mlp.forward_bf16(th, X.astype(np.float64))
    assert np.abs(out - ref).max() <= 2e-2 * np.abs(ref).max()
    # and the bf16 network is close to the exact one
    exact = mlp.forward(th, X.astype(np.float64))[0]
    assert np.abs(out - exact).max() <= 5e-2 * np.abs(exact).max()


def test_training_gradient_matches_oracle(model):
    th = _params(3)
    model.mlp_params(th)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((4099, 16)).astype(np.float32)
    Y = rng.standard_normal((4099, 3)).astype(np.float32)
    loss, g = model.mlp_grad(X, Y)
    # the tensor-core kernel's arithmetic: BF16 operands, FP32 accumulation
    ref_loss, ref_g = mlp.loss_grad_bf16(th, X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-4 * ref_loss
    assert np.linalg.norm(g - ref_g) <= 5e-3 * np.linalg.norm(ref_g)
    # and the exact FP64 backprop (itself pinned by finite differences)
    ex_loss, ex_g = mlp.loss_grad(th, X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - ex_loss) <= 2e-2 * ex_loss
    assert np.linalg.norm(g - ex_g) <= 3e-2 * np.linalg.norm(ex_g)


def test_learned_guess_gains_over_the_predictor(ctx):
    """The realistic model's layers and input on its 120 x 120 m lateral crop (106,875 DOF):
    500 training steps, then 200 steps with the learned guess on the Newmark predictor,
    against the same run with the plain predictor (the method without the network).  Both
    converge every step to relative residual 1e-8 and agree; the trained network stays
    active, lowers the initial residual at least twofold and needs no more outer
    iterations."""
    cfg = configs.config2(n_steps=700, crop=12)
    runs = {}
    for enable in (0, 1):
        m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
        m.set_time(cfg["dt"], cfg["n_steps"], cfg["band"])
        m.set_input(cfg["dir"], cfg["p"])
        m.set_solver(tol=1e-8, precision=2, inner_iters=30, guess_order=0)
        if enable:
            m.mlp_train(500, batch=16384, iters_per_step=2, lr=1e-3, seed=7)
            assert m.mlp_loss() > 0.0
        else:
            m.step(500)
        s0 = m.stats()
        m.step(200)
        s = m.stats()
        runs[enable] = dict(wave=m.waveforms(), iters=s["cg_iters_total"] - s0["cg_iters_total"],
                            r0=(s["init_relres_sum"] - s0["init_relres_sum"]) / 200, relres=s["relres_last"],
                            state=m.mlp_state() if enable else None)
        m.free()
    assert runs[0]["relres"] <= 1e-8 and runs[1]["relres"] <= 1e-8
    assert np.linalg.norm(runs[1]["wave"] - runs[0]["wave"]) <= 1e-6 * np.linalg.norm(runs[0]["wave"])
    st = runs[1]["state"]
    print("steps 501-700: outer iterations plain %d, learned %d; mean initial residual plain %.3e, learned %.3e; "
          "referee %s" % (runs[0]["iters"], runs[1]["iters"], runs[0]["r0"], runs[1]["r0"], st))
    assert st["active"] and st["learned_steps"] >= 150
    assert st["learned_r0"] < 0.5 * st["plain_r0"]
    assert runs[1]["r0"] < 0.5 * runs[0]["r0"]
    # on this crop two outer iterations per step suffice from either guess; on the full
    # model the same schedule takes 3.0 outer iterations per step to 2.1 (bench.py
    # --workload learned)
    assert runs[1]["iters"] <= runs[0]["iters"]


@pytest.mark.parametrize("order", [0, 2])
def test_learned_guess_data_path_matches_oracle(ctx, order):
    """Features, layer features, sampled training nodes, targets, base guess and output
    scale of the GPU's learned guess against the oracle's data path, both sides solving
    the same small box to relative residual 1e-11.  order 0: the network corrects the
    Newmark predictor; order 2: the quadratic extrapolation of the last three
    increments (output scale in both: the RMS of the previous step's correction)."""
    from oracle import fem
    from paper_2404_17754_gb300 import gsw

    cfg = configs.small_box(nx=4, ny=3, n_steps=12)
    n_run, B, seed, ips = 9, 256, 5, 2
    m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
    m.set_time(cfg["dt"], cfg["n_steps"], cfg["band"])
    m.set_input(cfg["dir"], cfg["p"])
    m.set_solver(tol=1e-11, precision=1, inner_iters=15, outer_op=gsw.OUTER_FP64, guess_order=order)
    m.set_learning(True, train_steps=100, batch=B, iters_per_step=ips, lr=1e-3, seed=seed)
    m.step(n_run)
    N = m.n_nodes
    nodes = np.arange(0, N, 7)
    got = m.mlp_inputs(nodes, B)
    m.free()

    ops = fem.assemble(cfg["mesh"], cfg["mat"], cfg["band"])
    C = (ops["CR"] + ops["Cabs"]).tocsr()
    w, dt = ops["w"][cfg["dir"]], cfg["dt"]
    z = np.zeros(3 * N)
    states = [(z, z, z)]
    newmark.newmark_run(ops["K"], ops["M"], C, lambda n: 2.0 * cfg["p"][n] * w, dt, n_run, tol=1e-11,
                        observe=lambda n, u, v, a: states.append((u.copy(), v.copy(), a.copy())))
    du = [states[k + 1][0] - states[k][0] for k in range(n_run)]
    nodef = mlp.layer_features(cfg["mesh"], cfg["mat"])

    def base_of(step):
        incs = [du[step - 1 - j] for j in range(step)]
        return mlp.base_guess(states[step][1], states[step][2], dt, incs, order).reshape(-1, 3)

    s = n_run - 1  # the last training step
    X_tr, sig = mlp.features([du[s - 1 - j] for j in range(4)], nodef)
    b_s = base_of(s)
    scale_s = mlp.correction_scale(du[s], b_s, sig[0])
    Y_tr = mlp.targets(du[s], b_s, scale_s)
    idx = mlp.sample_nodes(N, B, seed, s, ips - 1)
    assert np.abs(got["x_train"] - X_tr[idx]).max() <= 2e-5 * max(1.0, np.abs(X_tr[idx]).max())
    yr = np.sqrt(np.mean(Y_tr[idx] ** 2))
    assert np.abs(got["y_train"] - Y_tr[idx]).max() <= 1e-3 * yr
    # inputs of the next step's inference
    X_n, sig_n = mlp.features([du[s - j] for j in range(4)], nodef)
    b_n = base_of(s + 1)
    scale_n = mlp.correction_scale(du[s], b_s, sig_n[0])
    assert np.abs(got["x"] - X_n[nodes]).max() <= 2e-5 * max(1.0, np.abs(X_n[nodes]).max())
    assert np.abs(got["base"] - b_n[nodes]).max() <= 1e-8 * np.abs(b_n).max()
    assert abs(got["sigma"] - sig_n[0]) <= 1e-6 * sig_n[0]
    assert abs(got["scale"] - scale_n) <= 1e-4 * scale_n
