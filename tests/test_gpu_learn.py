"""GPU tests of the learned proposal (rows a10-a12): synthetic strain, patches,
the network's forward pass and gradient against the FP64 reference (with the
FP16-rounded weights the kernels multiply by), training, refinement against
the oracle and the full search, and the proposal search at its extremes."""
import numpy as np
import pytest

import oracle
import srs_synth
from oracle import mlp as omlp
from paper_2609_12476_gb300 import Context, Params
from paper_2609_12476_gb300 import proposal

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    c = Context(0)
    yield c
    c.close()


def test_make_strain_noise_is_standard_normal_and_seeded(ctx):
    from scipy import stats
    n = 1 << 22
    a = ctx.make_strain(n, 256.0, 11).cpu().numpy().astype(np.float64)
    b = ctx.make_strain(n, 256.0, 11).cpu().numpy()
    c = ctx.make_strain(n, 256.0, 12).cpu().numpy().astype(np.float64)
    assert np.array_equal(a.astype(np.float32), b)
    assert abs(a.mean()) < 5 / np.sqrt(n) and abs(a.var() - 1) < 5 * np.sqrt(2.0 / n)
    assert stats.kstest(a[:200000], "norm").pvalue > 1e-3
    assert abs(np.corrcoef(a, c)[0, 1]) < 5 / np.sqrt(n)
    assert abs(np.corrcoef(a[:-1], a[1:])[0, 1]) < 5 / np.sqrt(n)


def test_make_strain_chirp_matches_the_signal_model(ctx):
    fs, n = 256.0, 256 * 1200
    inj = {"mc": 0.1, "f0": 40.0, "amp": 0.5, "phi0": 0.3}
    x = ctx.make_strain(n, fs, 0, [inj], f_hi=60.0, noise=False).cpu().numpy().astype(np.float64)
    ref = srs_synth.chirp(n, fs, 0.1, 40.0, 0.5, 0.3)
    t_end = oracle.duration(oracle.beta(0.1, 40.0), 40.0, 60.0)     # 1060.5 s (Sec. V)
    j_end = int(np.ceil(t_end * fs))
    assert np.max(np.abs(x[:j_end - 1] - ref[:j_end - 1])) < 2e-6
    assert np.all(x[j_end + 1:] == 0.0)


def test_patches_match_the_reference(ctx):
    r = np.random.default_rng(0)
    smap = r.normal(0, 3, (20, 100)).astype(np.float32)
    cells = [(0, 0), (19, 99), (10, 50), (3, 97), (17, 2)]
    got = ctx.patches(smap, cells)
    ref = omlp.patches(smap.astype(np.float64), cells)
    assert np.max(np.abs(got - ref)) < 2e-6 * np.max(np.abs(ref))
    got_d = ctx.patches(torch.from_numpy(smap).cuda(), cells).cpu().numpy()
    assert np.array_equal(got_d, got)


def _case(seed, n):
    r = np.random.default_rng(seed)
    X = r.normal(0, 1, (n, omlp.D)).astype(np.float32)
    y = (r.random(n) < 0.5).astype(np.float32)
    p = proposal.init_params(seed)
    p[omlp.H * omlp.D:omlp.H * omlp.D + omlp.H] = r.normal(0, 0.1, omlp.H)
    p[-1] = 0.05
    return X, y, p


def test_forward_matches_reference_with_fp16_weights(ctx):
    X, _, p = _case(1, 300)
    got = ctx.mlp_forward(X, p)
    ref, _ = omlp.forward(X.astype(np.float64), omlp.fp16_weights(p))
    assert np.max(np.abs(got - ref)) <= 1e-4 * (1 + np.max(np.abs(ref)))


@pytest.mark.parametrize("shape", [(20, 600), (13, 130), (3, 40)])
def test_score_map_on_tensor_cores_matches_reference(ctx, shape):
    """Every cell's logit from the tensor-core scorer (implicit-GEMM first
    layer, FP16 features and weights, FP32 sums) against the FP64 network on
    the same FP16-rounded features and weights.  The shapes cover the map's
    edges (zero padding), a last tile of partial rows (600 = 4 x 128 + 88) and
    more tiles than SMs or fewer."""
    r = np.random.default_rng(11 + shape[0])
    smap = (r.normal(0, 2, shape) + 8 * (r.random(shape) < 0.01)).astype(np.float32)
    _, _, p = _case(4, 8)
    got = ctx.score_map(torch.from_numpy(smap).cuda(), p).cpu().numpy()
    cells = [(m, b) for m in range(shape[0]) for b in range(shape[1])]
    X = omlp.patches(smap.astype(np.float64), cells)
    X16 = X.astype(np.float16).astype(np.float64)
    p16 = omlp.fp16_weights(p)
    ref, _ = omlp.forward(X16, p16)
    W1, _, w2, _ = omlp.unpack(p16)
    # FP32 accumulation over 297 terms, and asinh in FP32 before the FP16 rounding
    # (one FP16 ulp, 2^-11 relative, where the two asinh round differently)
    bound = 2.0 ** -11 * (np.abs(X16) @ np.abs(W1).T) @ np.abs(w2) + 1e-5 * (1 + np.abs(ref))
    err = np.abs(got.ravel() - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


def test_gradient_matches_reference(ctx):
    X, y, p = _case(2, 257)
    g, loss = ctx.mlp_grad(X, y, p)
    p16 = omlp.fp16_weights(p)
    gr = omlp.grad(X.astype(np.float64), y.astype(np.float64), p16)
    assert loss == pytest.approx(omlp.loss(X.astype(np.float64), y.astype(np.float64), p16), rel=1e-5)
    assert np.linalg.norm(g - gr) <= 1e-4 * np.linalg.norm(gr)
    for sl in (slice(0, omlp.H * omlp.D), slice(omlp.H * omlp.D, None)):
        assert np.linalg.norm(g[sl] - gr[sl]) <= 1e-3 * np.linalg.norm(gr[sl])


def test_training_separates_bumps_from_noise(ctx):
    r = np.random.default_rng(3)
    n = 2048
    X = r.normal(0, 1, (n, omlp.T, omlp.B))
    y = (np.arange(n) % 2).astype(np.float32)
    X[y == 1, 3:6, 15:18] += 2.0
    X = np.arcsinh(X).reshape(n, omlp.D).astype(np.float32)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    torch.cuda.synchronize()
    p0 = proposal.init_params(4)
    p, losses = ctx.mlp_train(Xd, yd, p0, epochs=15, batch=128, lr=2e-3, seed=5)
    assert losses[-1] < 0.5 * losses[0]
    acc = np.mean((ctx.mlp_forward(X, p) > 0) == (y > 0.5))
    assert acc > 0.97


def _short_case():
    fs, T, n_seg = 256.0, 30.0, 8
    mc = srs_synth.log_templates(5e-2, 1e-1, 4)
    b3 = srs_synth.chirp_beta(mc[2], 40.0)
    x = srs_synth.strain_with_chirps(n_seg * 7680, fs, 9,
                                     [{"mc": srs_synth.mc_for_beta(b3, 47.0), "f0": 47.0, "amp": 0.1}])
    return x, mc


def test_refine_matches_oracle(ctx):
    x, mc = _short_case()
    p = Params(eps=1e-6)
    cells = [(2, 210), (2, 211), (0, 0), (3, 599), (1, 300), (2, 209)]
    ns, rep = ctx.refine(x, mc, p, cells)
    betas = [oracle.beta(m, 40.0) for m in mc]
    nsegs = [oracle.nseg(b, 40.0, 60.0, 30.0, 8) for b in betas]
    items = [(m, i) for m in range(len(mc)) for i in range(nsegs[m])]
    S, ref = oracle.semicoherent(x, 256.0, 30.0, 40.0, 600, betas, nsegs)
    for (m, b), v in zip(cells, ns):
        assert abs(v - ref[m, b]) <= 2e-5 * (1 + abs(ref[m, b])), (m, b, v, ref[m, b])
    assert ns[0] > 10     # the injected cell


def test_refine_agrees_with_the_full_search_map(ctx):
    w = srs_synth.make_workload("semicoherent_2h")
    p = Params(eps=1e-6)
    _, smap, _ = ctx.search(w["strain"], w["mc"], p)
    r = np.random.default_rng(7)
    cells = [(int(r.integers(64)), int(r.integers(600))) for _ in range(40)] + [(41, 149), (41, 150)]
    ns, _ = ctx.refine(w["strain"], w["mc"], p, cells)
    ref = np.array([smap[m, b] for m, b in cells])
    assert np.max(np.abs(ns - ref)) < 2e-3


def test_proposal_search_extremes(ctx):
    fs, nseg = 256.0, 24
    coarse = srs_synth.log_templates(3e-2, 1e-1, 6)
    fine = srs_synth.log_templates(3e-2, 1e-1, 24)
    x = srs_synth.strain_with_chirps(nseg * 7680, fs, 4, [{"mc": 6e-2, "f0": 50.0, "amp": 0.08}])
    p = Params(eps=1e-6, top_k=8)
    params = proposal.init_params(0)
    none = ctx.search_proposed(x, coarse, fine, p, params, threshold=np.inf, nms=(0, 0))
    assert none["n_cells"] == 0 and none["report"]["proposed_coarse"] == 0
    allc = ctx.search_proposed(x, coarse, fine, p, params, threshold=-np.inf, nms=(0, 0))
    assert allc["report"]["proposed_coarse"] == 6 * 600
    assert allc["n_cells"] == 24 * 600
    _, fmap, _ = ctx.search(x, fine, p)
    got = np.full(fmap.shape, np.nan, dtype=np.float32)
    got[allc["cells"][:, 0], allc["cells"][:, 1]] = allc["nsigma"]
    assert np.max(np.abs(got - fmap)) < 2e-3
    c = allc["cands"][0]
    assert c["value"] == pytest.approx(float(fmap.max()), abs=2e-3)


def test_proposal_suppression_keeps_local_maxima(ctx):
    fs, nseg = 256.0, 24
    coarse = srs_synth.log_templates(3e-2, 1e-1, 6)
    fine = srs_synth.log_templates(3e-2, 1e-1, 24)
    x = srs_synth.strain_with_chirps(nseg * 7680, fs, 4, [{"mc": 6e-2, "f0": 50.0, "amp": 0.08}])
    p = Params(eps=1e-6, top_k=8)
    params = proposal.init_params(0)
    r = ctx.search_proposed(x, coarse, fine, p, params, threshold=-np.inf, nms=(4, 16), fine_rows=0)
    smap = torch.from_numpy(ctx.search(x, coarse, p)[1]).cuda()
    sc = ctx.score_map(smap, params).cpu().numpy()
    assert r["report"]["proposed_coarse"] == int(proposal.peaks(sc, (4, 16)).sum())
    parent = [proposal.nearest_template(coarse, m) for m in fine]
    max_children = max(parent.count(c) for c in range(len(coarse)))
    assert 0 < r["n_cells"] <= r["report"]["proposed_coarse"] * max_children * 3


@pytest.mark.parametrize("top", [1, 3])
def test_proposal_component_rule_matches_host_rule(ctx, top):
    """component_top: the library proposes, per connected group of
    above-threshold cells, the `top` cells of highest coarse n_sigma -- the
    same cells as proposal.component_cells on the same maps."""
    fs, nseg = 256.0, 24
    coarse = srs_synth.log_templates(3e-2, 1e-1, 6)
    fine = srs_synth.log_templates(3e-2, 1e-1, 24)
    x = srs_synth.strain_with_chirps(nseg * 7680, fs, 4, [{"mc": 6e-2, "f0": 50.0, "amp": 0.08}])
    p = Params(eps=1e-6, top_k=8)
    params = proposal.init_params(0)
    smap = torch.from_numpy(ctx.search(x, coarse, p)[1]).cuda()
    sc = ctx.score_map(smap, params).cpu().numpy()
    th = float(np.float32(np.quantile(sc, 0.97)))
    keep = proposal.component_cells(sc, th, smap.cpu().numpy(), top)
    r = ctx.search_proposed(x, coarse, fine, p, params, threshold=th, fine_rows=0, component_top=top)
    assert r["report"]["proposed_coarse"] == int(keep.sum())
    expect = proposal.fine_cells_of(np.argwhere(keep), coarse, fine, 600, fine_rows=0)
    got = sorted(map(tuple, r["cells"].tolist()))
    assert got == [tuple(c) for c in expect]


@pytest.mark.parametrize("budget", [1, 5, 1000])
def test_proposal_template_budget_keeps_the_best_scored_templates(ctx, budget):
    """template_budget: only the fine templates whose best proposing coarse
    cell scores highest are refined; their cells are exactly the unbudgeted
    proposal's cells of those templates, with the same n_sigma.  A budget
    above the number of touched templates changes nothing."""
    fs, nseg = 256.0, 24
    coarse = srs_synth.log_templates(3e-2, 1e-1, 6)
    fine = srs_synth.log_templates(3e-2, 1e-1, 24)
    x = srs_synth.strain_with_chirps(nseg * 7680, fs, 4, [{"mc": 6e-2, "f0": 50.0, "amp": 0.08}])
    p = Params(eps=1e-6, top_k=8)
    params = proposal.init_params(0)
    smap = torch.from_numpy(ctx.search(x, coarse, p)[1]).cuda()
    sc = ctx.score_map(smap, params).cpu().numpy()
    th = float(np.float32(np.quantile(sc, 0.99)))
    full = ctx.search_proposed(x, coarse, fine, p, params, threshold=th, fine_rows=1)
    r = ctx.search_proposed(x, coarse, fine, p, params, threshold=th, fine_rows=1, template_budget=budget)
    kept = proposal.budget_templates(np.argwhere(sc > th), sc, coarse, fine, 1, budget)
    touched = {int(m) for m in full["cells"][:, 0]}
    assert len(kept) == min(budget, len(touched))
    want = {(int(m), int(b)): v for (m, b), v in zip(full["cells"], full["nsigma"]) if int(m) in kept}
    got = {(int(m), int(b)): v for (m, b), v in zip(r["cells"], r["nsigma"])}
    assert sorted(got) == sorted(want)
    assert r["report"]["proposed_coarse"] == full["report"]["proposed_coarse"]
    for c, v in got.items():
        assert v == pytest.approx(want[c], abs=2e-3)
    if budget >= len(touched):
        assert r["n_cells"] == full["n_cells"]
