"""GPU parity of the learned-proposal network (include/msp_learn.h) against the FP64 oracle
`oracle.proposal_oracle`, through the C ABI.

Bars.  A convolution's FP32 accumulation of exact BF16 x BF16 products, in any order, is within
K u32 sum|w x| of the exact sum (K terms, u32 = 2^-24): the building blocks are compared element
by element against that bound.  Through the network the BF16 roundings of the activations and
gradients amplify the accumulation error: where an FP32 result falls on the other side of a BF16
rounding boundary than the FP64 one, that value moves by one BF16 ulp.  The bar for the network
is measured from the oracle itself: four times the change of the result when every
pre-activation and pre-rounding gradient of the oracle is perturbed by noise of 2^-19 times its
RMS value (about sqrt(K) u32 for K = 576), plus 1e-5.
"""
import numpy as np
import pytest
import torch

from oracle import proposal_oracle as P

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
JIT = 2.0 ** -19


@pytest.fixture(scope="module")
def msp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_03902_gb300 import msp as m
    return m


def bf16_tensor(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)


@pytest.mark.parametrize("cin,cout", [(16, 64), (64, 64), (64, 16), (16, 16)])
@pytest.mark.parametrize("H,W", [(3, 256), (1, 128), (5, 384)])
def test_conv3x3_forward_matches_oracle(msp, cin, cout, H, W):
    rng = np.random.default_rng(100 + cin + cout + H)
    x = bf16_tensor(rng.standard_normal((H, W, cin)))
    w = (rng.standard_normal((cout, 9, cin)) / np.sqrt(9 * cin)).astype(np.float32)
    b = rng.standard_normal(cout).astype(np.float32)
    out, _ = msp.conv3x3_test(x.cuda(), torch.from_numpy(w).cuda(), torch.from_numpy(b).cuda())
    out = out.cpu().numpy().astype(np.float64)
    xo = x.to(torch.float64).numpy()
    wo = P.bf16(w)
    ref = P.conv3x3(xo, wo, b.astype(np.float64))
    absum = P.conv3x3(np.abs(xo), np.abs(wo)) + np.abs(b)
    bound = (9 * cin + 2) * U32 * absum
    err = np.abs(out - ref)
    assert np.all(err <= bound), (err.max(), bound[err > bound][:4])
    # without bias
    out0, _ = msp.conv3x3_test(x.cuda(), torch.from_numpy(w).cuda(), None)
    err0 = np.abs(out0.cpu().numpy() - P.conv3x3(xo, wo))
    assert np.all(err0 <= bound)


@pytest.mark.parametrize("cin,cout", [(16, 64), (64, 64), (64, 16), (16, 16)])
@pytest.mark.parametrize("H,W", [(3, 256), (2, 128)])
def test_conv3x3_weight_gradient_matches_oracle(msp, cin, cout, H, W):
    rng = np.random.default_rng(200 + cin + cout + H)
    x = bf16_tensor(rng.standard_normal((H, W, cin)))
    g = bf16_tensor(rng.standard_normal((H, W, cout)))
    dW, db, _ = msp.conv3x3_wgrad_test(x.cuda(), g.cuda())
    xo, go = x.to(torch.float64).numpy(), g.to(torch.float64).numpy()
    rW, rb = P.conv3x3_weight_grad(go, xo)
    aW, ab = P.conv3x3_weight_grad(np.abs(go), np.abs(xo))
    kW = (W + H + 2) * U32
    assert np.all(np.abs(dW.cpu().numpy() - rW) <= kW * aW)
    assert np.all(np.abs(db.cpu().numpy() - rb) <= (H * W + 2) * U32 * ab)


def _problem(L=4, H=64, W=256, seed=1):
    """Potential-like V (smooth, positive bumps), gradient-like G (signed, small), a target change."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    V = np.zeros((L, H, W))
    for l in range(L):
        for _ in range(12):
            cy, cx, r = rng.uniform(0, H), rng.uniform(0, W), rng.uniform(2, 6)
            V[l] += rng.uniform(0.5, 2.0) * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * r * r))
    G = 1e-3 * rng.standard_normal((L, H, W))
    T = 0.05 * rng.standard_normal((L, H, W))
    return V.astype(np.float32), G.astype(np.float32), T.astype(np.float32)


SCALES = dict(scale_v=1.0, scale_g=300.0, scale_d=0.05)


def _shape(msp, L, H, W):
    return msp.net_shape(L, H, W, **SCALES)


def test_net_init_is_bit_identical_to_the_oracle(msp):
    for L, seed in [(4, 3), (8, 12345678901234)]:
        p = msp.net_init(_shape(msp, L, 128, 128), seed).cpu().numpy()
        np.testing.assert_array_equal(p, P.init(L, seed))


def test_net_forward_matches_oracle(msp):
    L, H, W = 4, 64, 256
    V, G, _ = _problem(L, H, W)
    params = P.init(L, 5)
    params = params + np.float32(0.02) * np.random.default_rng(9).standard_normal(params.size).astype(np.float32)
    s = _shape(msp, L, H, W)
    out = msp.net_forward(s, torch.from_numpy(params).cuda(), torch.from_numpy(V).cuda(), torch.from_numpy(G).cuda())
    out = out.cpu().numpy()
    sc = (SCALES["scale_v"], SCALES["scale_g"], SCALES["scale_d"])
    ref = P.proposal(params, L, V, G, *sc)
    sens = max(np.linalg.norm(P.proposal(params, L, V, G, *sc, jitter=(np.random.default_rng(k), JIT)) - ref)
               for k in (1, 2)) / np.linalg.norm(ref)
    bar = 4 * sens + 1e-5
    rel = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert rel <= bar, (rel, bar)


def _loss_grad_case(msp, L, H, W, seed):
    V, G, T = _problem(L, H, W, seed)
    params = P.init(L, seed)
    params = params + np.float32(0.02) * np.random.default_rng(seed).standard_normal(params.size).astype(np.float32)
    sc = (SCALES["scale_v"], SCALES["scale_g"], SCALES["scale_d"])
    loss_o, grad_o, mags = P.loss_and_grad(params, L, V, G, T, *sc, abs_sums=True)
    jit = [P.loss_and_grad(params, L, V, G, T, *sc, jitter=(np.random.default_rng(k), JIT)) for k in (1, 2)]
    return V, G, T, params, loss_o, grad_o, jit, mags


@pytest.mark.parametrize("L,H,W", [(4, 64, 256), (2, 7, 128)])
def test_net_loss_grad_matches_oracle(msp, L, H, W):
    V, G, T, params, loss_o, grad_o, jit, _ = _loss_grad_case(msp, L, H, W, seed=L + H)
    s = _shape(msp, L, H, W)
    d = lambda a: torch.from_numpy(a).cuda()
    loss, grad = msp.net_loss_grad(s, d(params), d(V), d(G), d(T))
    grad = grad.cpu().numpy().astype(np.float64)
    loss_bar = 4 * max(abs(l - loss_o) for l, _ in jit) / loss_o + 1e-6
    assert abs(loss.item() - loss_o) / loss_o <= loss_bar
    for i, (ci, co, wo, bo) in enumerate(P.layout(L)):
        for lo, hi, what in [(wo, bo, "weights"), (bo, bo + co, "biases")]:
            ref = grad_o[lo:hi]
            sens = max(np.linalg.norm(gj[lo:hi] - ref) for _, gj in jit) / np.linalg.norm(ref)
            rel = np.linalg.norm(grad[lo:hi] - ref) / np.linalg.norm(ref)
            assert rel <= 4 * sens + 1e-5, (i, what, rel, sens)


def test_net_train_step_is_adam_on_the_oracle_gradient(msp):
    """Adam's first step moves every parameter by lr g / (|g| + 1e-8).  The gradient error allowed
    per entry is eight times the spread of the perturbed oracles (the BF16 rounding flips) plus the
    accumulation error of its sum over the H W pixels: the weight-gradient kernel sums each image
    row on the tensor core, then the rows in order, the bias gradient sums all pixels.  The tensor
    core's FP32 accumulation aligns the addends of a block to the largest exponent and truncates
    (measured on NVIDIA tensor cores by Fasi, Higham, Mikaitis and Pranesh, PeerJ Comput. Sci.
    2021), so the round-to-nearest bound (W + H + 2) u32 sum_p |g| |x| does not hold entry by
    entry: up to 3.6 times it was seen on entries whose sum cancels; the test allows 8 times.
    Where the gradient is more than twice the allowed error from zero its sign is fixed and the
    step must match; everywhere the step is at most lr."""
    L, H, W = 4, 64, 256
    V, G, T, params, loss_o, grad_o, jit, mags = _loss_grad_case(msp, L, H, W, seed=21)
    s = _shape(msp, L, H, W)
    d = lambda a: torch.from_numpy(a).cuda()
    p = d(params.copy())
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    lr = 1e-3
    loss = msp.net_train_step(s, p, m, v, 1, lr, d(V), d(G), d(T))
    step = p.cpu().numpy().astype(np.float64) - params.astype(np.float64)
    p_o, _, _ = P.adam(params.astype(np.float64), 0.0, 0.0, grad_o, 1, lr)
    step_o = p_o - params.astype(np.float64)
    spread = np.max([np.abs(gj - grad_o) for _, gj in jit], axis=0)
    acc = np.full(params.size, 8 * (W + H + 2) * U32)
    for ci, co, wo, bo in P.layout(L):
        acc[bo:bo + co] = (H * W + 2) * U32
    e_g = 8 * spread + acc * mags + 1e-7 * np.abs(grad_o).max()      # the gradient error allowed
    sure = np.abs(grad_o) > 2 * e_g
    assert sure.mean() > 0.5
    # the step's FP32 arithmetic, the FP32 storage of p, and the step's sensitivity to the gradient
    # through eps: d/dg [g / (|g| + eps)] = eps / (|g| + eps)^2
    tol = 1e-5 * lr + 4 * U32 * np.abs(params.astype(np.float64))
    tol_sure = tol + lr * 1e-8 * e_g / (np.abs(grad_o) - e_g) ** 2
    bad = (np.abs(step - step_o) > tol_sure) & sure
    if bad.any():
        _, g_c = msp.net_loss_grad(s, d(params), d(V), d(G), d(T))
        g_c = g_c.cpu().numpy().astype(np.float64)
        idx = np.nonzero(bad)[0]
        where = []
        for i in idx[:6]:
            for k, (ci, co, wo, bo) in enumerate(P.layout(L)):
                if wo <= i < bo + co:
                    where.append((int(i), k, "bias" if i >= bo else "weight"))
        raise AssertionError(f"{bad.sum()} entries: (index, layer, is_bias) {where}; oracle g {grad_o[idx][:6]}; "
                             f"cuda g {g_c[idx][:6]}; spread {spread[idx][:6]}; acc {(acc * mags)[idx][:6]}; "
                             f"max|g| {np.abs(grad_o).max()}")
    assert np.all(np.abs(step) <= lr * (1 + 1e-5) + tol)
    assert abs(loss.item() - loss_o) / loss_o < 1e-3


def test_training_reduces_the_loss_on_a_fixed_batch(msp):
    """A learnable target (a local function of the input: a scaled copy of the potentials minus the
    gradients) on one image: a hundred Adam steps must halve the loss."""
    L, H, W = 4, 64, 256
    V, G, _ = _problem(L, H, W, seed=3)
    T = (0.02 * V - 10.0 * G).astype(np.float32)
    s = _shape(msp, L, H, W)
    d = lambda a: torch.from_numpy(a).cuda()
    p = msp.net_init(s, 4)
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    ws = msp.net_make_workspace(s)
    losses = [msp.net_train_step(s, p, m, v, k, 1e-3, d(V), d(G), d(T), ws=ws).item() for k in range(1, 101)]
    msp.check_workspace(ws)
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])


def test_conv_wait_that_runs_out_is_reported(msp):
    """With no poll allowed (msp_set_wait_limit(-1)) every convolution's first wait for its MMAs
    gives up: the kernel stops, waits for the MMAs it issued and frees its tensor memory; the
    call's workspace reads MSP_ETIMEOUT and the same process runs the network correctly
    afterwards.  (With a bound of one poll the waits succeed: each CTA waits for the MMAs of a row
    only after staging the next input row.)"""
    L, H, W = 2, 64, 256
    V, G, T = _problem(L, H, W, seed=5)
    s = _shape(msp, L, H, W)
    d = lambda a: torch.from_numpy(a).cuda()
    p = msp.net_init(s, 1)
    ws = msp.net_make_workspace(s)
    timed_out = False
    try:
        msp.set_wait_limit(-1)
        for _ in range(3):
            msp.net_forward(s, p, d(V), d(G), ws=ws)
            try:
                msp.check_workspace(ws)
            except msp.MspError as e:
                assert e.status == msp.MSP_ETIMEOUT
                timed_out = True
                break
    finally:
        msp.set_wait_limit(0)
    assert timed_out
    out = msp.net_forward(s, p, d(V), d(G), ws=ws).cpu().numpy()
    msp.check_workspace(ws)
    ref = P.proposal(p.cpu().numpy(), L, V, G, SCALES["scale_v"], SCALES["scale_g"], SCALES["scale_d"])
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-2


def test_weight_gradient_wait_that_runs_out_is_reported(msp):
    """The backward pass under msp_set_wait_limit(-1): every tensor-core kernel of it, the
    weight-gradient kernel's tensor-load producer and MMA thread included, gives up at its first
    wait, drains what it issued with its own fixed bound and frees its tensor memory; the
    workspace reads MSP_ETIMEOUT and the next call's loss and gradient are right."""
    L, H, W = 2, 64, 256
    V, G, T = _problem(L, H, W, seed=6)
    s = _shape(msp, L, H, W)
    d = lambda a: torch.from_numpy(a).cuda()
    p = msp.net_init(s, 2)
    ws = msp.net_make_workspace(s)
    timed_out = False
    try:
        msp.set_wait_limit(-1)
        for _ in range(3):
            msp.net_loss_grad(s, p, d(V), d(G), d(T), ws=ws)
            try:
                msp.check_workspace(ws)
            except msp.MspError as e:
                assert e.status == msp.MSP_ETIMEOUT
                timed_out = True
                break
    finally:
        msp.set_wait_limit(0)
    assert timed_out
    loss, grad = msp.net_loss_grad(s, p, d(V), d(G), d(T), ws=ws)
    msp.check_workspace(ws)
    sc = (SCALES["scale_v"], SCALES["scale_g"], SCALES["scale_d"])
    loss_o, grad_o = P.loss_and_grad(p.cpu().numpy(), L, V, G, T, *sc)
    assert abs(loss.item() - loss_o) / loss_o < 1e-2
    g = grad.cpu().numpy()
    assert np.linalg.norm(g - grad_o) / np.linalg.norm(grad_o) < 5e-2
