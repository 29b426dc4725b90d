"""Learned proposal: training data, training, calibration and the recall reference.

Host orchestration of the library's kernels (every computation runs in
libsrs: strain synthesis, searches, patches, the network, refinement):

  training_set  seeded strain realisations with 0PN chirps injected on a
                grid of well-separated coarse cells (amplitudes uniform in a
                range) -> the coarse search -> 9 x 33 patches centred (with
                +-1 jitter) on injection cells (label 1) and on cells far from
                any injection (label 0), in equal shares
  init_params   a seeded Kaiming-uniform start for the 297-64-1 network
  train         Adam on the device set
  calibrate     score threshold that proposes a fraction `far` of the cells of
                noise-only coarse maps (and the same for coarse n_sigma, the
                proposal without a network)
  evaluate      recall of injections: full fine-template search vs the
                proposal search vs the n_sigma-threshold proposal, at a per-cell
                false-alarm probability from the exact chi^2 null of the
                equal-weight statistic (Sec. III.C: n_sigma is an affine map of
                chi^2 with 2 N_seg degrees of freedom)
"""
import math

import numpy as np

from . import _capi
from ._capi import Params, SRS_F32

GMSUN_C3 = 1.32712440018e20 / 299792458.0 ** 3


def beta_of(mc, f):
    """Sec. II Eq. (beta)."""
    return (96.0 / 5.0) * math.pi ** (8.0 / 3.0) * (GMSUN_C3 * mc) ** (5.0 / 3.0) * f ** (8.0 / 3.0)


def log_bank(lo, hi, n):
    return np.exp(np.linspace(np.log(lo), np.log(hi), n))


def nearest_template(bank, mc):
    return int(np.argmin(np.abs(np.log(bank) - np.log(mc))))


def injections_on_grid(rng, coarse_mc, params, count, amp_range, t_rows=9, b_cols=33):
    """`count` injections on distinct cells of a (t_rows x b_cols)-spaced grid
    of the coarse map, so their patches do not overlap.  Each injection's
    chirp parameter at its f0 equals a template chirp parameter at f_ref
    somewhere inside its cell (label mass log-uniform within the cell, f0
    uniform within the bin).  Returns (injections, cells)."""
    n_bins = int(round((params.f_hi - params.f_lo) * params.t_coh))
    M = len(coarse_mc)
    rows = list(range(t_rows // 2, M - t_rows // 2, t_rows))
    cols = list(range(b_cols // 2, n_bins - b_cols // 2, b_cols))
    slots = [(r, c) for r in rows for c in cols]
    pick = rng.choice(len(slots), size=min(count, len(slots)), replace=False)
    dlog = np.log(coarse_mc[1] / coarse_mc[0]) if M > 1 else 0.1
    inj, cells = [], []
    for k in pick:
        m, b = slots[k]
        label = coarse_mc[m] * math.exp(rng.uniform(-0.5, 0.5) * dlog)
        f0 = params.f_lo + (b + rng.uniform(-0.5, 0.5)) / params.t_coh
        # beta(f0, mc_inj) = beta(f_ref, label)  =>  mc_inj = label (f_ref / f0)^(8/5)
        mc_inj = label * (params.f_ref / f0) ** 1.6
        amp = rng.uniform(*amp_range)
        inj.append({"mc": mc_inj, "f0": f0, "amp": amp, "phi0": rng.uniform(0, 2 * math.pi), "label": label})
        cells.append((m, b))
    return inj, cells


def coarse_map(ctx, strain, coarse_mc, params):
    out = {"map": None, "cands": None}
    import torch
    M = len(coarse_mc)
    n_bins = int(round((params.f_hi - params.f_lo) * params.t_coh))
    out["map"] = torch.empty((M, n_bins), dtype=torch.float32, device=strain.device)
    out["cands"] = torch.empty((params.top_k, 3), dtype=torch.int32, device=strain.device)
    res, rep = ctx.search(strain, coarse_mc, params, out=out)
    return res["map"], rep


def training_set(ctx, coarse_mc, params, t_obs, n_real, per_real, seed, amp_range=(0.01, 0.1)):
    """Device tensors X [N, 297], y [N] from n_real realisations.  Per
    injection: its cell with the centre jittered by up to one template and one
    bin (label 1) and a near miss two to four templates or two to twelve bins
    away (label 0); plus twice as many patches of cells far from every injection
    (label 0) -- half the patches from injection regions, half pure noise."""
    import torch
    rng = np.random.default_rng(seed)
    n = int(round(t_obs * params.fs))
    n_bins = int(round((params.f_hi - params.f_lo) * params.t_coh))
    M = len(coarse_mc)
    Xs, ys = [], []
    for r in range(n_real):
        inj, cells = injections_on_grid(rng, coarse_mc, params, per_real, amp_range)
        x = ctx.make_strain(n, params.fs, seed * 1000003 + r, inj, f_hi=params.f_hi)
        smap, _ = coarse_map(ctx, x, coarse_mc, params)
        pos = [(min(M - 1, max(0, m + rng.integers(-1, 2))), min(n_bins - 1, max(0, b + rng.integers(-1, 2))))
               for m, b in cells]
        near = []
        for m, b in cells:
            if rng.random() < 0.5:
                dm, db = int(rng.choice([-1, 1]) * rng.integers(2, 5)), int(rng.integers(-1, 2))
            else:
                dm, db = int(rng.integers(-1, 2)), int(rng.choice([-1, 1]) * rng.integers(2, 13))
            near.append((min(M - 1, max(0, m + dm)), min(n_bins - 1, max(0, b + db))))
        taken = np.zeros((M, n_bins), dtype=bool)
        for m, b in cells:
            taken[max(0, m - 6):m + 7, max(0, b - 20):b + 21] = True
        free = np.argwhere(~taken)
        neg = [tuple(free[k]) for k in rng.choice(len(free), size=2 * len(pos), replace=False)]
        X = ctx.patches(smap, pos + near + neg)
        Xs.append(X)
        ys.append(torch.tensor([1.0] * len(pos) + [0.0] * (len(near) + len(neg)), dtype=torch.float32,
                               device=X.device))
    return torch.cat(Xs), torch.cat(ys)


def hard_negatives(ctx, mlp_params, coarse_mc, params, t_obs, n_maps, per_map, seed):
    """The highest-scoring cells of pure-noise coarse maps, as label-0 patches."""
    import torch
    Xs = []
    for smap in noise_maps(ctx, coarse_mc, params, t_obs, n_maps, seed):
        sc = ctx.score_map(smap, mlp_params).flatten()
        top = torch.topk(sc, per_map).indices.cpu().numpy()
        nb = smap.shape[1]
        Xs.append(ctx.patches(smap, [(int(c) // nb, int(c) % nb) for c in top]))
    X = torch.cat(Xs)
    return X, torch.zeros(X.shape[0], dtype=torch.float32, device=X.device)


def train_proposal(ctx, coarse_mc, params, t_obs, n_patches=20000, per_real=64, seed=1, hard_frac=0.25,
                   epochs=(30, 20, 10), lrs=(1e-3, 3e-4, 1e-4), batch=256):
    """The full training recipe: n_patches patches, half injections (amplitude
    uniform in [0.01, 0.1]) and half pure noise, of which hard_frac come from
    the top scores of pure-noise maps after a first round.  Returns
    (parameters, per-epoch losses, held-out (X, y))."""
    import torch
    n_neg_hard = int(n_patches * 0.5 * hard_frac)
    n_real = int(math.ceil((n_patches - n_neg_hard) / (4.0 * per_real)))
    X, y = training_set(ctx, coarse_mc, params, t_obs, n_real, per_real, seed)
    g = torch.Generator().manual_seed(seed)
    perm = torch.randperm(X.shape[0], generator=g).to(X.device)
    n_hold = max(1, X.shape[0] // 10)
    Xh, yh = X[perm[:n_hold]].contiguous(), y[perm[:n_hold]].contiguous()
    Xt, yt = X[perm[n_hold:]].contiguous(), y[perm[n_hold:]].contiguous()
    torch.cuda.synchronize()
    p = init_params(seed)
    losses = []
    p, l = ctx.mlp_train(Xt, yt, p, epochs=epochs[0], batch=batch, lr=lrs[0], seed=seed)
    losses += list(l)
    if n_neg_hard > 0:
        per_map = 512
        Xn, yn = hard_negatives(ctx, p, coarse_mc, params, t_obs, max(1, n_neg_hard // per_map), per_map, seed + 17)
        Xt, yt = torch.cat([Xt, Xn]).contiguous(), torch.cat([yt, yn]).contiguous()
        torch.cuda.synchronize()
    for e, lr in zip(epochs[1:], lrs[1:]):
        p, l = ctx.mlp_train(Xt, yt, p, epochs=e, batch=batch, lr=lr, seed=seed + e)
        losses += list(l)
    return p, np.array(losses), (Xh, yh), int(Xt.shape[0])


def init_params(seed):
    """Kaiming-uniform weights (fan-in), zero biases."""
    r = np.random.default_rng(seed)
    D, H = _capi.MLP_INPUTS, _capi.MLP_HIDDEN
    p = np.zeros(_capi.MLP_PARAMS, dtype=np.float32)
    p[:H * D] = r.uniform(-1, 1, H * D) * math.sqrt(6.0 / D)
    p[H * D + H:H * D + 2 * H] = r.uniform(-1, 1, H) * math.sqrt(6.0 / H)
    return p


def noise_maps(ctx, coarse_mc, params, t_obs, n_maps, seed):
    n = int(round(t_obs * params.fs))
    for r in range(n_maps):
        x = ctx.make_strain(n, params.fs, seed * 7919 + r, [], f_hi=params.f_hi)
        yield coarse_map(ctx, x, coarse_mc, params)[0]


NMS = (4, 16)        # suppression half-window: the patch's half-size (templates, bins)
NO_NMS = (0, 0)      # default: every cell above threshold is proposed (suppression costs recall
                     # when injections crowd a map: a loud ridge hides its neighbours' peaks)


def peaks(values, nms):
    """Mask of the cells that are the maximum of their (+-nms[0], +-nms[1])
    window (ties: the first in row-major order keeps it)."""
    from scipy.ndimage import maximum_filter
    v = np.asarray(values, dtype=np.float64)
    if nms[0] <= 0 and nms[1] <= 0:
        return np.ones(v.shape, dtype=bool)
    mx = maximum_filter(v, size=(2 * nms[0] + 1, 2 * nms[1] + 1), mode="constant", cval=-np.inf)
    return v >= mx


def component_cells(score, threshold, nsigma, top):
    """Mask of the cells the component rule proposes (the library's
    srs_search_proposed with component_top = top): of each 8-connected group of
    cells whose score exceeds the threshold, the `top` cells of highest coarse
    n_sigma (ties: lower row-major index first)."""
    from scipy.ndimage import label
    score = np.asarray(score)
    mask = score > threshold
    lab, n = label(mask, structure=np.ones((3, 3), dtype=int))
    keep = np.zeros(score.shape, dtype=bool)
    if n == 0:
        return keep
    idx = np.flatnonzero(mask)
    grp = lab.ravel()[idx]
    ns = np.asarray(nsigma, dtype=np.float32).ravel()[idx]
    order = np.lexsort((idx, -ns, grp))
    g = grp[order]
    start = np.r_[0, np.flatnonzero(np.diff(g)) + 1]
    rank = np.arange(len(g)) - np.repeat(start, np.diff(np.r_[start, len(g)]))
    keep.ravel()[idx[order[rank < top]]] = True
    return keep


def _threshold_for_count(maps, k, component_top):
    """Score threshold whose component-rule proposals over `maps` ((score,
    n_sigma) pairs) number about k: the first threshold, scanning scores
    downwards by bisection, at which at least k cells are proposed."""
    vals = np.sort(np.concatenate([s.ravel() for s, _ in maps]))[::-1]
    count = lambda t: sum(int(component_cells(s, t, n, component_top).sum()) for s, n in maps)
    lo, hi = 0, len(vals) - 1
    while lo < hi:
        mid = (lo + hi) // 2
        if count(vals[mid]) >= k:
            hi = mid
        else:
            lo = mid + 1
    return float(vals[lo])


def calibrate(ctx, mlp_params, coarse_mc, params, t_obs, n_maps, seed, far, nms=NO_NMS, component_top=0,
              nms_by_nsigma=False):
    """Thresholds that propose a fraction `far` of the cells of pure-noise coarse
    maps (after non-maximum suppression -- on the score, or on the coarse
    n_sigma with nms_by_nsigma -- or under the component rule): one on the
    network's score, one on the coarse n_sigma (the proposal without a
    network)."""
    sc_peaks, ns_peaks, total, maps = [], [], 0, []
    for smap in noise_maps(ctx, coarse_mc, params, t_obs, n_maps, seed):
        sc = ctx.score_map(smap, mlp_params).double().cpu().numpy()
        ns = smap.double().cpu().numpy()
        total += sc.size
        if component_top > 0:
            maps.append((sc.astype(np.float32), ns.astype(np.float32)))
        else:
            sc_peaks.append(sc[peaks(ns if nms_by_nsigma else sc, nms)])
            ns_peaks.append(ns[peaks(ns, nms)])
    k = max(1, int(round(far * total)))
    if component_top > 0:
        return (_threshold_for_count(maps, k, component_top),
                _threshold_for_count([(n, n) for _, n in maps], k, component_top))
    sp = np.sort(np.concatenate(sc_peaks))[::-1]
    npk = np.sort(np.concatenate(ns_peaks))[::-1]
    return float(sp[min(k, len(sp) - 1)]), float(npk[min(k, len(npk) - 1)])


def detection_threshold(nseg, p_fa):
    """n_sigma threshold at per-cell false-alarm probability p_fa:
    n_sigma = (S - 2N) / (2 sqrt N) with S ~ chi^2_{2N} under noise."""
    from scipy.stats import chi2
    nseg = np.asarray(nseg, dtype=np.float64)
    return (chi2.isf(p_fa, 2 * nseg) - 2 * nseg) / (2 * np.sqrt(nseg))


def evaluate(ctx, mlp_params, score_th, nsigma_th, coarse_mc, fine_mc, params, t_obs, n_real, per_real, seed,
             p_fa=1e-6, amp_range=(0.01, 0.1), nms=NO_NMS, fine_rows=1, component_top=0, nms_by_nsigma=False,
             plain_subset=False, baselines=True, template_budget=0):
    """Recall of injections over the same realisations in these searches:
      full            every fine template (the recall reference), mixed form
      proposal        the network's proposal at its noise-calibrated threshold
                      (the library's srs_search_proposed)
      nsigma_equal    the proposal without the network at equal cost: the same
                      number of coarse cells, the highest coarse n_sigma first
      nsigma_far      the proposal without the network at the same noise false-
                      alarm rate: coarse cells above the calibrated n_sigma threshold
      plain_fp64      (plain_subset) the plain FP64 form of the full search on
                      the fine templates within +-2 of each injection's own,
                      the only templates that decide its recall
    An injection counts as recovered when a cell within +-2 fine templates and
    +-1 bin of its own (label) cell exceeds the detection threshold at
    per-cell false-alarm probability p_fa; in the proposal searches that cell
    must also have been evaluated.  baselines=False skips the two searches
    without the network; template_budget > 0 caps the fine templates the
    proposal refines (srs_proposal_params.template_budget)."""
    import torch
    rng = np.random.default_rng(seed)
    n = int(round(t_obs * params.fs))
    n_bins = int(round((params.f_hi - params.f_lo) * params.t_coh))
    Mf = len(fine_mc)
    info, _, nseg_f = _capi.srs_plan(params, fine_mc, n)
    th_f = detection_threshold(nseg_f, p_fa)
    keys = ("full", "proposal") + (("nsigma_equal", "nsigma_far") if baselines else ()) + \
        (("plain_fp64",) if plain_subset else ())
    out = {"injections": 0, "full_ms": 0.0, "proposal_ms": 0.0, "full_spectra": 0, "proposal_coarse_spectra": 0,
           "proposal_segment_bins": 0, "proposed_coarse": 0, "plain_ms": 0.0, "plain_spectra": 0,
           "plain_mixed_max_dnsigma": 0.0}
    for k in keys:
        out[k] = 0
        out[k + "_cells"] = 0
    for r in range(n_real):
        inj, _cells = injections_on_grid(rng, coarse_mc, params, per_real, amp_range)
        x = ctx.make_strain(n, params.fs, seed * 1000003 + 7 + r, inj, f_hi=params.f_hi)
        # full fine search (the recall reference)
        fmap = torch.empty((Mf, n_bins), dtype=torch.float32, device=x.device)
        res, rep = ctx.search(x, fine_mc, params, out={"map": fmap, "cands": torch.empty((params.top_k, 3),
                              dtype=torch.int32, device=x.device)})
        out["full_ms"] += rep["device_ms"]
        out["full_spectra"] += rep["n_spectra"]
        fm = fmap.cpu().numpy()
        found = {"full": {(m, b): float(fm[m, b]) for m, b in np.argwhere(fm > th_f[:, None])}}
        out["full_cells"] += fm.size
        # the network's proposal search
        pr = ctx.search_proposed(x, coarse_mc, fine_mc, params, mlp_params, score_th, nms=nms, fine_rows=fine_rows,
                                 component_top=component_top, nms_by_nsigma=nms_by_nsigma,
                                 template_budget=template_budget)
        out["proposal_ms"] += pr["report"]["device_ms"]
        out["proposal_coarse_spectra"] += pr["report"]["coarse_spectra"]
        out["proposal_segment_bins"] += pr["report"]["fine_segment_bins"]
        out["proposed_coarse"] += pr["report"]["proposed_coarse"]
        out["proposal_cells"] += pr["n_cells"]
        found["proposal"] = {(int(m), int(b)): float(v) for (m, b), v in zip(pr["cells"], pr["nsigma"])}
        if plain_subset:
            # the plain FP64 form on the templates that decide recall
            sub = sorted({m for I in inj for m in range(max(0, nearest_template(fine_mc, I["label"]) - 2),
                                                        min(Mf, nearest_template(fine_mc, I["label"]) + 3))})
            pp = Params(**{f: getattr(params, f) for f in params.__dataclass_fields__})
            pp.precision = _capi.SRS_PLAIN_FP64
            pmap = torch.empty((len(sub), n_bins), dtype=torch.float32, device=x.device)
            _, prep = ctx.search(x, fine_mc[sub], pp, out={"map": pmap, "cands": torch.empty(
                (params.top_k, 3), dtype=torch.int32, device=x.device)})
            out["plain_ms"] += prep["device_ms"]
            out["plain_spectra"] += prep["n_spectra"]
            pm = pmap.cpu().numpy()
            out["plain_mixed_max_dnsigma"] = max(out["plain_mixed_max_dnsigma"],
                                                 float(np.max(np.abs(pm - fm[sub]))))
            found["plain_fp64"] = {(sub[r], int(b)): float(pm[r, b]) for r, b in np.argwhere(pm > th_f[sub][:, None])}
        if not baselines:
            for I in inj:
                out["injections"] += 1
                mf = nearest_template(fine_mc, I["label"])
                bf = int(round((I["f0"] - params.f_lo) * params.t_coh))
                nb = [(m, b) for m in range(max(0, mf - 2), min(Mf, mf + 3))
                      for b in range(max(0, bf - 1), min(n_bins, bf + 2))]
                for key in keys:
                    if any(found[key].get((m, b), -np.inf) > th_f[m] for m, b in nb):
                        out[key] += 1
            continue
        # proposals without the network
        cmap, _ = coarse_map(ctx, x, coarse_mc, params)
        cm = cmap.cpu().numpy()
        K = pr["report"]["proposed_coarse"]
        if component_top > 0:
            # the same rule on the n_sigma map: K cells at the threshold that
            # first proposes K, and the cells above the calibrated threshold
            t_eq = _threshold_for_count([(cm, cm)], K, component_top) if K > 0 else np.inf
            eq = np.argwhere(component_cells(cm, t_eq, cm, component_top))
            eq = eq[np.argsort(-cm[eq[:, 0], eq[:, 1]], kind="stable")[:K]]
            far_cells = np.argwhere(component_cells(cm, nsigma_th, cm, component_top))
        else:
            pk = peaks(cm, nms)
            cand = np.argwhere(pk)
            eq = cand[np.argsort(-cm[pk])[:K]]
            far_cells = np.argwhere(pk & (cm > nsigma_th))
        for key, prop in (("nsigma_equal", eq), ("nsigma_far", far_cells)):
            fc = fine_cells_of(prop, coarse_mc, fine_mc, n_bins, fine_rows)
            out[key + "_cells"] += len(fc)
            found[key] = {}
            if len(fc):
                nsb, _ = ctx.refine(x, fine_mc, params, fc)
                found[key] = {(int(m), int(b)): float(v) for (m, b), v in zip(fc, nsb)}
        for I in inj:
            out["injections"] += 1
            mf = nearest_template(fine_mc, I["label"])
            bf = int(round((I["f0"] - params.f_lo) * params.t_coh))
            nb = [(m, b) for m in range(max(0, mf - 2), min(Mf, mf + 3))
                  for b in range(max(0, bf - 1), min(n_bins, bf + 2))]
            for key in keys:
                if any(found[key].get((m, b), -np.inf) > th_f[m] for m, b in nb):
                    out[key] += 1
    for key in keys:
        out["recall_" + key] = out[key] / max(1, out["injections"])
    return out


def budget_templates(coarse_cells, scores, coarse_mc, fine_mc, fine_rows, budget):
    """The fine templates a template budget keeps: each fine template touched
    by a proposed coarse cell ranks by the best score among the cells that
    touch it (ties: lower index first); the first `budget` are kept."""
    parent = np.array([nearest_template(coarse_mc, m) for m in fine_mc])
    best = {}
    for m, b in coarse_cells:
        s = float(scores[int(m), int(b)])
        for f in np.nonzero(np.abs(parent - int(m)) <= fine_rows)[0]:
            best[int(f)] = max(best.get(int(f), -np.inf), s)
    order = sorted(best, key=lambda f: (-best[f], f))
    return set(order[:budget])


def fine_cells_of(coarse_cells, coarse_mc, fine_mc, n_bins, fine_rows=1):
    """Fine (template, bin) cells proposed by coarse cells: fine templates whose
    nearest coarse template is within fine_rows of the cell's, bins within one."""
    parent = np.array([nearest_template(coarse_mc, m) for m in fine_mc])
    children = {}
    for f, c in enumerate(parent):
        children.setdefault(int(c), []).append(f)
    cells = set()
    for m, b in coarse_cells:
        for c in range(int(m) - fine_rows, int(m) + fine_rows + 1):
            for f in children.get(c, []):
                for bb in range(max(0, int(b) - 1), min(n_bins, int(b) + 2)):
                    cells.add((f, bb))
    return sorted(cells)
