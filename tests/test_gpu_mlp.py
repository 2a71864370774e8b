"""Learned CG initial guess on the GPU against the CPU oracle of the MLP.

* tensor-core (BF16 operands, FP32 accumulation) inference vs the oracle's
  bf16-rounded forward pass;
* FP32 training gradients vs the oracle's FP64 analytic backprop (itself
  pinned by finite differences);
* a run that trains on its first steps and then applies the guess converges
  every step to the same 1e-8 relative residual and reproduces the plain run;
  the guess quality (initial residual) and CG iterations are compared.
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
    ref_loss, ref_g = mlp.loss_grad(th, X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    assert np.linalg.norm(g - ref_g) <= 1e-4 * np.linalg.norm(ref_g)


def test_learned_guess_run_converges_and_matches_plain(ctx):
    from paper_2404_17754_gb300 import gsw

    cfg = configs.config1(n_steps=120)
    runs = {}
    for enable in (0, 1):
        m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
        m.set_time(cfg["dt"], cfg["n_steps"], cfg["band"])
        m.set_input(cfg["dir"], cfg["p"])
        m.set_solver(tol=1e-8, precision=1, inner_iters=15)
        if enable:
            m.set_learning(True, train_steps=60, batch=4096, iters_per_step=4, lr=2e-3, seed=5)
        it_train = None
        m.step(60)
        s60 = m.stats()
        if enable:
            assert m.mlp_loss() > 0.0
        m.step(60)
        s = m.stats()
        runs[enable] = dict(wave=m.waveforms(), iters=s["cg_iters_total"] - s60["cg_iters_total"],
                            r0=(s["init_relres_sum"] - s60["init_relres_sum"]) / 60, relres=s["relres_last"],
                            state=m.mlp_state() if enable else None)
        m.free()
    assert runs[1]["relres"] <= 1e-8
    rel = np.linalg.norm(runs[1]["wave"] - runs[0]["wave"]) / np.linalg.norm(runs[0]["wave"])
    assert rel <= 1e-6
    ref = newmark.analysis(cfg, tol=1e-8)["wave"]
    assert np.linalg.norm(runs[1]["wave"] - ref) / np.linalg.norm(ref) <= 1e-6
    st = runs[1]["state"]
    print("outer iterations over steps 61-120: plain %d, learned %d; mean initial residual: plain %.3e, learned "
          "%.3e; judge: %s" % (runs[0]["iters"], runs[1]["iters"], runs[0]["r0"], runs[1]["r0"], st))
    assert st["learned_steps"] >= 5
    # the judge keeps the learned guess only while it beats the plain predictor
    if st["active"]:
        assert st["learned_r0"] <= st["plain_r0"]
    else:
        assert st["learned_steps"] < 60
    # and the run as a whole is not made much worse than the plain one
    assert runs[1]["iters"] <= 1.2 * runs[0]["iters"]
