"""Learned format selector: the library's MLP kernels against the fp64 reference,
the GPU column statistics against their plain definition, and the trained
selector's regret against the exhaustive try-all-formats choice."""
import numpy as np
import pytest
import torch

from oracle import mlp
from paper_2004_09350_gb300 import morphstore as ms
from paper_2004_09350_gb300 import selector, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.random((n, 16)).astype(np.float32)
    y = rng.normal(size=(n, 10)).astype(np.float32)
    m = (rng.random((n, 10)) < 0.9).astype(np.float32)
    return x, y, m


def test_mlp_forward_matches_reference():
    theta = mlp.init(1).astype(np.float32)
    x, _, _ = _data(1000, 2)
    got = ms.mlp_forward(torch.from_numpy(theta).to(DEV), torch.from_numpy(x).to(DEV)).cpu().numpy()
    want, _ = mlp.forward(theta.astype(np.float64), x.astype(np.float64))
    np.testing.assert_allclose(got, want, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("n", [1, 37, 3000])
def test_mlp_gradient_matches_reference(n):
    theta = mlp.init(3).astype(np.float32)
    x, y, m = _data(n, 4)
    inv = 1.0 / max(m.sum(), 1.0)
    grad = torch.zeros(ms.MLP_PARAMS, device=DEV)
    loss = torch.zeros(1, device=DEV)
    parts = torch.zeros(700 * (ms.MLP_PARAMS + 1), device=DEV)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    ms.mlp_loss_grad(t(theta), t(x), t(y), t(m), inv, grad, loss, parts)
    L, g = mlp.loss_grad(theta.astype(np.float64), x, y, m, inv)
    assert abs(float(loss.item()) - L) <= 1e-4 * abs(L) + 1e-7
    got = grad.cpu().numpy()
    scale = np.abs(g).max()
    np.testing.assert_allclose(got, g, rtol=1e-3, atol=1e-4 * scale)
    # deterministic: the same call gives the same bits
    grad2 = torch.zeros_like(grad)
    ms.mlp_loss_grad(t(theta), t(x), t(y), t(m), inv, grad2, loss, parts)
    assert torch.equal(grad, grad2)


@pytest.mark.parametrize("steps", [1, 5])
def test_mlp_adam_matches_reference(steps):
    # The library's Adam kernel (fp32) against the fp64 Adam of oracle/mlp.py, element by
    # element after every step: parameters, first and second moments.  Each reference
    # step starts from the GPU's current state, so fp32 rounding does not compound.
    # Tolerance: the fp32 rounding bound of each update.  m = b1*m + (1-b1)*g can
    # cancel, so its bound is relative to the two terms, not to the result:
    # |err| <= 3 * 2^-24 * (|b1*m| + |(1-b1)*g|); v has no cancellation (2^-22
    # relative); theta - step rounds once and the step carries about a dozen
    # roundings (the fp32 bias corrections, divisions, square root, products):
    # 2^-23*|theta| + 12*2^-24*|step|.
    rng = np.random.default_rng(8)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)
    dth, dm, dv = t(mlp.init(9)), t(np.zeros(mlp.PARAMS)), t(np.zeros(mlp.PARAMS))
    # the kernel takes its hyperparameters as fp32: the reference uses those exact values
    lr, b1, b2, eps = (float(np.float32(a)) for a in (3e-3, 0.9, 0.999, 1e-8))
    u = 2.0 ** -24
    for step in range(1, steps + 1):
        g = rng.normal(scale=10.0 ** float(rng.integers(-4, 2)), size=mlp.PARAMS).astype(np.float32)
        th0, m0, v0 = [a.cpu().numpy().astype(np.float64) for a in (dth, dm, dv)]
        want = mlp.adam_step(th0, g, m0, v0, step, lr, b1, b2, eps)
        ms.mlp_adam(dth, t(g), dm, dv, step, lr=lr, beta1=b1, beta2=b2, eps=eps)
        torch.cuda.synchronize()
        got = [a.cpu().numpy().astype(np.float64) for a in (dth, dm, dv)]
        g64 = g.astype(np.float64)
        bound_m = 3 * u * (np.abs(b1 * m0) + np.abs((1 - b1) * g64)) + 1e-38
        assert (np.abs(got[1] - want[1]) <= bound_m).all(), np.max(np.abs(got[1] - want[1]) / bound_m)
        np.testing.assert_allclose(got[2], want[2], rtol=4 * u, atol=1e-38)
        step_size = np.abs(th0 - want[0])
        bound_t = 2 * u * np.abs(want[0]) + 12 * u * step_size + 1e-38
        assert (np.abs(got[0] - want[0]) <= bound_t).all(), np.max(np.abs(got[0] - want[0]) / bound_t)


def test_mlp_training_reduces_loss():
    x, _, _ = _data(2000, 5)
    # a learnable target: fixed random linear map of the features
    w = np.random.default_rng(6).normal(size=(16, 10))
    y = (x @ w).astype(np.float32)
    sel = selector.Selector(DEV, seed=7)
    hist = sel.train(x, y, epochs=300, lr=3e-3)
    assert hist[-1][1] < 0.1 * hist[0][1]


def _plain_stats(x):
    n = x.size
    st = np.zeros(80, dtype=np.uint64)
    st[0] = n
    if n == 0:
        return st
    st[1] = x.max()
    for c in range(0, n, 512):
        blk = x[c:c + 512].astype(object)
        st[2] += 1
        st[3] += (max(blk) - min(blk)).bit_length()
        d = [(blk[i] - blk[i - 1]) % 2**64 for i in range(1, len(blk))]
        st[4] += (max(d) if d else 0).bit_length()
        st[5] += sum(1 for i in range(1, len(blk)) if blk[i] >= blk[i - 1])
        st[6] += sum(1 for i in range(1, len(blk)) if blk[i] != blk[i - 1])
        st[8 + max(blk).bit_length()] += 1
    return st


@pytest.mark.parametrize("fmt", [ms.UNCOMPR, ms.DYN_BP, ms.DELTA_BP])
@pytest.mark.parametrize("kind", ["skewed", "sorted", "C2"])
def test_column_stats_match_plain_definition(fmt, kind):
    n = 6 * 512 + 77
    x = {"skewed": synth.skewed_widths(1, n), "sorted": synth.sorted_gaps(2, n),
         "C2": synth.table1_column("C2", n)}[kind]
    with ms.Ctx(0, arena_bytes=64 << 20, max_rows=n) as ctx:
        col = ctx.compress(ms.as_device_u64(x, DEV), fmt)
        got = ctx.column_stats(col).cpu().numpy().view(np.uint64)
        ctx.check()
    np.testing.assert_array_equal(got, _plain_stats(x))


def test_selector_regret_against_exhaustive_choice():
    with ms.Ctx(0, arena_bytes=1 << 30, max_rows=1 << 20) as ctx:
        items = list(selector.synthetic_intermediates(11, 330, lo_log2=14, hi_log2=18))
        X, Y, S, T, names = selector.harvest(ctx, items, reps=1)
    rng = np.random.default_rng(0)
    idx = rng.permutation(len(X))
    tr, te = idx[:264], idx[264:]
    sel = selector.Selector(DEV, seed=1)
    sel.train(X[tr], Y[tr], epochs=600, lr=3e-3)
    chosen = sel.choose(X[te], "size")
    r = selector.regret(chosen, S[te])
    static_all = selector.regret(np.full(len(te), ms.STATIC_BP), S[te])
    best_fixed = min(selector.regret(np.full(len(te), f), S[te]) for f in range(5))
    assert r <= 0.05, r
    assert r < static_all and r < best_fixed, (r, static_all, best_fixed)
    # run-time labels: at 2^14-2^18 rows and one timed repetition the formats' times differ
    # by a few percent and carry timing noise, so the regret is bounded rather than required
    # to beat every fixed format (the 2e4-trace bench measures it on longer columns)
    rt = selector.regret(sel.choose(X[te], "time"), T[te])
    assert 0.0 <= rt <= 0.05, rt
