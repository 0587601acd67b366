"""The learned surrogate on the GPU (tcgen05 training and inference kernels) against its FP64
oracle: gradients, the fused inference kernel, and distillation from a forest."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_1811_00156_gb300 import synth
from tests.mlp_cases import model, violations

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


def _model(A, seed=0, n=512):
    P, X, mu, sd, lg, y = model(seed, n)
    return P, X, mu, sd, lg, y, A.aiwcrf_surrogate_create(32, 15, 4, P, mu, sd, lg)


def test_gradient_matches_fp64_oracle(A):
    """Every one of the 82,689 gradient entries, and the loss, lie within the oracle's
    element-wise tolerance (oracle/mlp.py grad_tolerance). The tolerance is a running error
    analysis of the device's arithmetic: FP32 operations err by at most u = 2^-24 relative;
    log2f, erff and expf by at most 1, 2 and 2 ulp; a K-term FP32 accumulation of exact BF16
    products by at most 2 K u times the sum of the absolute terms; GELU and GELU' move by their
    Taylor bounds under an argument error; and a value known within E rounds to BF16 within
    bf16(v + E) - bf16(v - E) of the oracle's rounded value. The bounds propagate through the
    forward pass, the loss and the backward pass as the device computes them. The CPU tests show
    it admits an independent float32 evaluation and rejects planted mistakes, among them a 5 %
    error in one W2 gradient entry."""
    P, X, mu, sd, lg, y, sg = _model(A)
    n = X.shape[1]
    g = torch.empty(M.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    sg.grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), g, loss)
    torch.cuda.synchronize()
    rl, rg, lb, gb = M.grad_tolerance(P.astype(np.float64), X, mu, sd, lg, 15, 4, y.astype(np.float64))
    assert abs(float(loss.item()) - rl) <= lb, (float(loss.item()), rl, lb)
    v = violations(g.cpu().numpy(), rg, gb)
    assert all(c == 0 for c, _ in v.values()), v
    assert n == 512


# The inference epilogues evaluate erf by Abramowitz & Stegun formula 7.1.26 (absolute error at
# most 1.5e-7) with the approximate reciprocal and exponential. Their FP32 evaluation adds at most
# about 9.4e-7 more: the reciprocal's relative error (2^-22 on t, through a polynomial of slope
# <= 2), five FMA roundings on partial sums below 1.5, the exponential's relative error (2^-22)
# and its argument's two roundings (2u x^2 e^(-x^2) <= 0.74u), and the final FMA. 2e-6 covers it.
ERF_INFER_ERR = 2e-6


def test_fused_inference_matches_oracle_forward(A):
    """Every prediction of the fused inference kernel lies within the oracle's element-wise
    tolerance of the rounded forward pass (oracle/mlp.py forward_tolerance, the same running
    error analysis as the gradient's, with the epilogues' erf error)."""
    P, _, mu, sd, lg, _, sg = _model(A, seed=5)
    for Q in (1, 127, 128, 1000, 70001):
        X = synth.queries(Q, seed=Q)
        out = torch.empty(Q, dtype=torch.float32, device="cuda")
        sg.predict(torch.from_numpy(X).cuda(), out)
        torch.cuda.synchronize()
        ref, bound = M.forward_tolerance(P.astype(np.float64), X, mu, sd, lg, 15, 4, erf_err=ERF_INFER_ERR)
        err = np.abs(out.cpu().numpy().astype(np.float64) - ref)
        assert np.all(err <= bound), (Q, int(np.sum(err > bound)), float(np.max(err / bound)))


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
