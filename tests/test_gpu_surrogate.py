"""The learned surrogate on the GPU (tcgen05 training and inference kernels) against its FP64
oracle: gradients, the fused inference kernel, and distillation from a forest."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_1811_00156_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1811_00156_gb300 import aiwcrf
    return aiwcrf


def _model(A, seed=0):
    rng = np.random.default_rng(seed)
    P = rng.normal(0.0, 0.08, M.N_PARAMS).astype(np.float32)
    P[M.OW1:M.OB1].reshape(M.HID, M.K_IN)[:, 49:] = 0.0
    P[M.OB3] = -2.0
    mu = rng.normal(0.0, 1.0, 30).astype(np.float32)
    sd = rng.uniform(0.5, 3.0, 30).astype(np.float32)
    lg = np.zeros(30, np.uint8)
    lg[:10] = 1
    lg[24:] = 1
    return P, mu, sd, lg, A.aiwcrf_surrogate_create(32, 15, 4, P, mu, sd, lg)


def test_gradient_matches_fp64_oracle(A):
    P, mu, sd, lg, sg = _model(A)
    n = 512
    X = synth.queries(n, seed=3)
    y = np.random.default_rng(4).normal(-3.0, 1.0, n).astype(np.float32)
    g = torch.empty(M.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    sg.grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), g, loss)
    torch.cuda.synchronize()
    xin = M.encode(X, mu, sd, lg, 15, 4)
    rl, rg = M.loss_and_grad(P.astype(np.float64), xin, y.astype(np.float64))
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - rl) <= 1e-3 * abs(rl)
    for name, a, b in [("W1", M.OW1, M.OB1), ("b1", M.OB1, M.OW2), ("W2", M.OW2, M.OB2), ("b2", M.OB2, M.OW3),
                       ("w3", M.OW3, M.OB3), ("b3", M.OB3, M.N_PARAMS)]:
        rel = np.linalg.norm(gg[a:b] - rg[a:b]) / (np.linalg.norm(rg[a:b]) + 1e-30)
        assert rel < 2e-2, (name, rel)


def test_fused_inference_matches_oracle_forward(A):
    P, mu, sd, lg, sg = _model(A, seed=5)
    for Q in (1, 127, 128, 1000, 70001):
        X = synth.queries(Q, seed=Q)
        out = torch.empty(Q, dtype=torch.float32, device="cuda")
        sg.predict(torch.from_numpy(X).cuda(), out)
        torch.cuda.synchronize()
        ref, _ = M.forward(P.astype(np.float64), M.encode(X, mu, sd, lg, 15, 4))
        err = np.abs(out.cpu().numpy() - ref)
        assert err.max() <= 2e-2 * (np.abs(ref).max() + 1.0), (Q, err.max())
        assert np.median(err) <= 2e-3 * (np.abs(ref).max() + 1.0)


def test_distillation_learns_the_forest(A):
    wl = synth.plain_forest_workload()
    forest = A.aiwcrf_fit(A.params(64, 10, 5), torch.from_numpy(wl.X).cuda(), torch.from_numpy(wl.y).cuda())
    Xs = torch.from_numpy(synth.queries(131072, seed=11)).cuda()
    sg = A.aiwcrf_surrogate_fit(A.surrogate_params(epochs=6, batch=4096), forest, Xs)
    st = sg.stats()
    assert st["steps"] == 6 * 32 and st["last_batch_loss"] < 0.5 * st["first_batch_loss"]
    Xt = synth.queries(20000, seed=12)
    ref = torch.empty(20000, dtype=torch.int64, device="cuda")
    A.aiwcrf_predict(forest, torch.from_numpy(Xt).cuda(), ref)
    out = torch.empty(20000, dtype=torch.float32, device="cuda")
    sg.predict(torch.from_numpy(Xt).cuda(), out)
    torch.cuda.synchronize()
    f = ref.cpu().numpy() / 2.0 ** 32
    s = out.cpu().numpy().astype(np.float64)
    mae = np.abs(s - f).mean()
    base = np.abs(f - f.mean()).mean()                   # predicting the mean, without the network
    assert mae < 0.5 * base, (mae, base)
