"""Host-side rules of the learned proposal (paper_2609_12476_gb300.proposal)
against brute force: local-maximum suppression, the fine cells a coarse cell
proposes, injections placed on the coarse grid, and the detection threshold.
CPU only."""
import math

import numpy as np
import pytest

from paper_2609_12476_gb300 import Params, nsigma_threshold, proposal


def test_peaks_against_brute_force():
    r = np.random.default_rng(5)
    v = r.integers(0, 7, size=(13, 29)).astype(np.float64)     # many ties
    for nms in ((1, 2), (4, 16), (0, 3), (0, 0)):
        got = proposal.peaks(v, nms)
        want = np.zeros_like(got)
        for m in range(v.shape[0]):
            for b in range(v.shape[1]):
                win = v[max(0, m - nms[0]):m + nms[0] + 1, max(0, b - nms[1]):b + nms[1] + 1]
                want[m, b] = v[m, b] >= win.max()
        assert np.array_equal(got, want), nms


def test_fine_cells_against_brute_force():
    coarse = proposal.log_bank(5e-4, 1e-1, 16)
    fine = proposal.log_bank(5e-4, 1e-1, 64)
    n_bins = 40
    cells = [(0, 0), (7, 20), (15, 39), (8, 21)]
    for rows in (0, 1, 2):
        got = set(map(tuple, proposal.fine_cells_of(cells, coarse, fine, n_bins, fine_rows=rows)))
        want = set()
        for f, mc in enumerate(fine):
            parent = int(np.argmin(np.abs(np.log(coarse) - np.log(mc))))
            for m, b in cells:
                if abs(parent - m) <= rows:
                    want.update((f, bb) for bb in (b - 1, b, b + 1) if 0 <= bb < n_bins)
        assert got == want, rows


def test_injections_on_grid_sit_in_their_cells():
    """Each injection's chirp parameter at its f0 equals the chirp parameter of
    its label mass at f_ref (Sec. II Eq. beta), the label lies within half a
    template step of its cell's template, f0 within half a bin of the cell's
    bin, and no two cells' patches overlap."""
    p = Params()
    coarse = proposal.log_bank(5e-4, 1e-1, 256)
    rng = np.random.default_rng(9)
    inj, cells = proposal.injections_on_grid(rng, coarse, p, 40, (0.01, 0.1))
    assert len(inj) == 40 and len(set(cells)) == 40
    step = math.log(coarse[1] / coarse[0])
    for i, (m, b) in zip(inj, cells):
        assert proposal.beta_of(i["mc"], i["f0"]) == pytest.approx(proposal.beta_of(i["label"], p.f_ref), rel=1e-12)
        assert abs(math.log(i["label"] / coarse[m])) <= 0.5 * step + 1e-12
        assert abs((i["f0"] - p.f_lo) * p.t_coh - b) <= 0.5 + 1e-9
        assert 0.01 <= i["amp"] <= 0.1
    for a in range(len(cells)):
        for c in range(a + 1, len(cells)):
            (m1, b1), (m2, b2) = cells[a], cells[c]
            assert abs(m1 - m2) >= 9 or abs(b1 - b2) >= 33


def test_detection_threshold_matches_the_library():
    for n in (1, 35, 240, 720):
        assert proposal.detection_threshold(n, 1e-6) == pytest.approx(nsigma_threshold(n, 1e-6), rel=1e-9)


def test_budget_templates_against_brute_force():
    """The template budget's host restatement: a fine template ranks by the
    best score of the proposed coarse cells whose rows (within fine_rows of
    its nearest coarse template) touch it; ties go to the lower index."""
    rng = np.random.default_rng(3)
    coarse = np.geomspace(1e-2, 1e-1, 7)
    fine = np.geomspace(1e-2, 1e-1, 29)
    scores = rng.integers(0, 5, size=(7, 40)).astype(np.float32)   # many ties
    cells = np.argwhere(scores >= 3)
    parent = [int(np.argmin(np.abs(np.log(coarse) - np.log(m)))) for m in fine]
    for rows in (0, 1):
        best = {}
        for m, b in cells:
            for f in range(len(fine)):
                if abs(parent[f] - m) <= rows:
                    best[f] = max(best.get(f, -np.inf), scores[m, b])
        ranked = sorted(best, key=lambda f: (-best[f], f))
        for budget in (1, 4, 11, 100):
            got = proposal.budget_templates(cells, scores, coarse, fine, rows, budget)
            assert got == set(ranked[:budget]), (rows, budget)
    # a row that no proposed cell reaches contributes nothing
    only = np.array([[0, 5]])
    got = proposal.budget_templates(only, scores, coarse, fine, 0, 100)
    assert got == {f for f in range(len(fine)) if parent[f] == 0}
