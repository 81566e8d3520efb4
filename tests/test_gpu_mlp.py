"""The learned-guess perceptron: device FP32 kernels against the FP64 oracle MLP, and training on
solutions the method produces."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2512_13550_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_mlp_loss_and_gradient_match_oracle():
    from paper_2512_13550_gb300 import learned
    F, H, O, B = 8, 256, 1, 300
    net = learned.MLP(F, H, O, seed=2)
    theta = net.theta.double().cpu().numpy()
    X = inputs.normal(21, B * F).reshape(B, F)
    T = inputs.normal(22, B * O).reshape(B, O)
    loss_ref, g_ref = omlp.loss_and_grad(theta, X, T, F, H, O)
    Xt = torch.tensor(X, dtype=torch.float32, device="cuda")
    Tt = torch.tensor(T, dtype=torch.float32, device="cuda")
    loss = learned.mlp_loss_grad(net, Xt, Tt)
    torch.cuda.synchronize()
    assert abs(loss.item() - loss_ref) < 1e-5 * max(1.0, loss_ref)
    g = net.grad.double().cpu().numpy()
    assert np.max(np.abs(g - g_ref)) < 1e-5 * max(1.0, np.max(np.abs(g_ref)))
    Y = learned.mlp_forward(net, Xt).double().cpu().numpy()
    np.testing.assert_allclose(Y, omlp.forward(theta, X, F, H, O)[0], rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("wd", [0.0, 0.3])
def test_mlp_adam_step_matches_definition(wd):
    """Bias-corrected Adam (Kingma & Ba) with decoupled weight decay, first step."""
    from paper_2512_13550_gb300 import learned
    net = learned.MLP(4, 16, 1, seed=5)
    th0 = net.theta.double().cpu().numpy()
    net.grad.copy_(torch.tensor(inputs.normal(30, net.P), dtype=torch.float32, device="cuda"))
    g = net.grad.double().cpu().numpy()
    learned.mlp_adam(net, lr=1e-2, wd=wd)
    torch.cuda.synchronize()
    m = 0.1 * g
    v = 0.001 * g * g
    ref = th0 - 1e-2 * ((m / 0.1) / (np.sqrt(v / 0.001) + 1e-8) + wd * th0)
    np.testing.assert_allclose(net.theta.double().cpu().numpy(), ref, rtol=1e-5, atol=1e-6)


def test_learned_guess_trains_on_method_solutions():
    """Occupations the method converges to are learnable from the pair features: the held-out error
    of the trained network is well below that of predicting the training mean."""
    from paper_2512_13550_gb300 import learned
    orb, aux = inputs.basis_3s_10aux()
    Xtr, ytr = learned.generate(inputs.batch_sizes(120, seed=21, lo=6, hi=24), orb, aux, seed=11)
    Xte, yte = learned.generate(inputs.batch_sizes(16, seed=22, lo=6, hi=24), orb, aux, seed=12)
    assert 0.0 <= ytr.min() and ytr.max() <= 1.0 + 1e-12
    net = learned.MLP(learned.NFEAT, 256, 1, seed=0)
    hist = learned.train(net, Xtr, ytr, iters=800, lr=1e-3, wd=0.3)
    assert hist[-1] < 0.3 * hist[0]
    pred = learned.predict(net, Xte)
    err = np.sqrt(np.mean((pred - yte) ** 2))
    base = np.sqrt(np.mean((ytr.mean() - yte) ** 2))
    assert err < 0.7 * base
    # the learned start is a valid occupation guess (angles in [0, pi/2])
    g0 = learned.angles(pred)
    assert np.all(g0 >= 0) and np.all(g0 <= np.pi / 2 + 1e-12)


def test_bf16_inference_matches_oracle_forward():
    """BF16 tensor-core inference (mma.sync, FP32 accumulation) against the FP64 oracle forward
    pass: inputs, activations and weights rounded to BF16 (relative 2^-9 each) give outputs
    within 2e-2 of the output scale, and the same network's FP32 forward agrees at that level."""
    from paper_2512_13550_gb300 import learned
    F, H, O, B = 8, 256, 2, 333  # a ragged batch: 21 tiles of 16 rows, the last one partial
    net = learned.MLP(F, H, O, seed=4)
    theta = net.theta.double().cpu().numpy()
    X = inputs.normal(41, B * F).reshape(B, F)
    ref = omlp.forward(theta, X, F, H, O)[0]
    bnet = learned.BF16Net(net)
    net.mu, net.sd = np.zeros(F), np.ones(F)
    Y = bnet(X)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(Y - ref)) < 2e-2 * scale
    assert np.max(np.abs(Y - ref)) > 0.0  # it is a BF16 computation, not the FP32 path
    Y32 = learned.mlp_forward(net, torch.tensor(X, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    assert np.max(np.abs(Y32 - ref)) < 1e-5 * scale


@pytest.mark.slow
def test_learned_start_from_converged_solutions_saves_evaluations():
    """Trained on 300 converged solutions of displaced H6-H40 chains (occupations and pair rotation
    angles from nof_optimize), the BF16 network's start converges on held-out H24, H40 and H64 to
    the core guess's minimum or a lower one, in fewer evaluations in total; the start with the
    automatic fallback converges too. The rows (E_start, E_final, iterations, evaluations per start)
    are printed."""
    from paper_2512_13550_gb300 import learned
    orb, aux = inputs.basis_3s_10aux()
    X, T, recs = learned.converged_solutions(inputs.batch_sizes(300, seed=21, lo=6, hi=40), orb, aux, seed=31)
    assert all(r[3] for r in recs)
    net = learned.MLP(learned.NFEAT, 256, learned.NOUT, seed=0)
    hist = learned.train(net, X, T, iters=1500, lr=1e-3, wd=0.3)
    assert hist[-1] < 0.5 * hist[0]
    rows = learned.compare_starts(learned.BF16Net(net), [24, 40, 64], orb, aux)
    for r in rows:
        print(r)
        for name in ("core", "learned", "learned_occupations", "learned_or_core"):
            assert r[name]["converged"], (r["N"], name)
        assert r["learned"]["E_final"] <= r["core"]["E_final"] + 1e-6
    ev = {name: sum(r[name]["evaluations"] for r in rows) for name in ("core", "learned", "learned_occupations")}
    print("evaluations to ||g|| < 1e-4 over H24, H40, H64:", ev)
    assert ev["learned"] < ev["core"]
