"""The batched ensemble at its real candidate sizes.

Eight seeded candidates of the FP64 ensemble (config-1 box, soft-layer depth
Gaussian random fields, 35..62 lateral cells: 0.5-3 M DOF each, uneven) run
together as one batch in the plain FP64 form (block-Jacobi PCG, every
iteration in the step graph's device-side loop).  At these sizes the oracle
checks sampled outputs: operator rows at sampled nodes against the oracle
assembled from only the elements and faces touching them, and the true
Newmark residual of the batched steps, f - (M a + C v + K u) at t_{n+1},
relative to the step's right-hand side (<= 2e-8 at tolerance 1e-8).
"""
import numpy as np
import pytest

from oracle import fem
from synth import configs

pytestmark = pytest.mark.gpu


def test_real_size_fp64_batch_rows_and_true_residual():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_17754_gb300 import build, gsw
    from test_gpu_parity import _sampled_rows

    build.build()
    ctx = gsw.Context(0)
    rng = np.random.default_rng(12)
    cfgs = [configs.config3_candidate(l, n_steps=3) for l in range(8)]
    dofs = [3 * c["mesh"]["xyz"].shape[0] for c in cfgs]
    assert min(dofs) >= 4e5 and max(dofs) <= 3.2e6 and len(set(dofs)) > 1
    models = []
    for cfg in cfgs:
        m = ctx.upload(cfg["mesh"], cfg["mat"], cfg["rec_xy"])
        m.set_time(cfg["dt"], 3, cfg["band"])
        m.set_input(cfg["dir"], cfg["p"])
        m.set_solver(tol=1e-8, precision=0)
        models.append(m)
    tt = lambda a: torch.tensor(a, device="cuda")
    # sampled operator rows of every candidate against the oracle
    for cfg, m in zip(cfgs, models):
        nodes = rng.choice(m.n_nodes, 12, replace=False)
        ops = _sampled_rows(cfg["mesh"], cfg["mat"], cfg["band"], nodes)
        dt = cfg["dt"]
        A = ops["K"] + (2 / dt) * (ops["CR"] + ops["Cabs"]) + (4 / dt ** 2) * ops["M"]
        x = rng.standard_normal((m.n_nodes, 3))
        rows = (3 * nodes[:, None] + np.arange(3)).ravel()
        y = m.apply(0, tt(x)).cpu().numpy().ravel()[rows]
        ref = (A @ x.ravel())[rows]
        assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)
    b = ctx.batch(models)
    b.step(2)
    states0 = [m.get_state() for m in models]
    b.step(1)
    b.close()
    for cfg, m, (u0, v0, a0, k0) in zip(cfgs, models, states0):
        u1, v1, a1, k1 = m.get_state()
        assert k0 == 2 and k1 == 3 and m.stats()["relres_last"] <= 1e-8
        mesh = cfg["mesh"]
        base_faces = mesh["face_tag"] == 1
        base = fem.assemble(dict(mesh, conn=mesh["conn"][:1], elem_mat=mesh["elem_mat"][:1],
                                 faces=mesh["faces"][base_faces],
                                 face_elem=np.zeros(int(base_faces.sum()), dtype=np.int32),
                                 face_tag=mesh["face_tag"][base_faces]),
                            np.repeat(cfg["mat"][-1:], cfg["mat"].shape[0], axis=0), cfg["band"])
        f = 2.0 * cfg["p"][2] * base["w"][cfg["dir"]]
        lhs = (m.apply(2, tt(a1)) + m.apply(3, tt(v1)) + m.apply(1, tt(u1))).cpu().numpy().ravel()
        res = f - lhs
        rhs = m.apply(0, tt(u1 - u0)).cpu().numpy().ravel() + res
        rel = np.linalg.norm(res) / np.linalg.norm(rhs)
        assert rel <= 2e-8, rel
        m.free()
    print("real-size FP64 batch: DOF %s" % dofs)
    ctx.close()
