"""The learned proposal end to end on the GPU, at reduced size: training data
made by the search itself, training by the library's kernels, calibration at
a 1e-3 noise false-alarm rate, and the recall reference (the full fine-template
search).  With many loud injections per map the coarse n_sigma map is full of
ridges; the network must still find the injections' own cells, and beat the
proposal without a network given the same number of coarse cells."""
import numpy as np
import pytest

from paper_2609_12476_gb300 import Context, Params, proposal

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_proposal_recall_and_gain_over_no_network():
    ctx = Context(0)
    p = Params(eps=1e-6, top_k=16)
    coarse = proposal.log_bank(5e-4, 1e-1, 256)
    fine = proposal.log_bank(5e-4, 1e-1, 4096)
    t_obs = 7200.0
    params, losses, (Xh, yh), n_tr = proposal.train_proposal(ctx, coarse, p, t_obs, n_patches=8000, seed=3,
                                                             epochs=(30, 15, 10))
    assert losses[-1] < losses[0]
    lh = ctx.mlp_forward(Xh, params).cpu().numpy()
    yy = yh.cpu().numpy()
    pos, neg = lh[yy > 0.5], lh[yy < 0.5]
    auc = (pos[:, None] > neg[None, :]).mean()
    assert auc > 0.85
    sth, nth = proposal.calibrate(ctx, params, coarse, p, t_obs, 4, seed=5, far=1e-3)
    ev = proposal.evaluate(ctx, params, sth, nth, coarse, fine, p, t_obs, 2, 64, seed=11)
    ctx.close()
    print(ev)
    assert ev["recall_full"] > 0.8
    assert ev["recall_proposal"] >= 0.7 * ev["recall_full"]
    assert ev["recall_proposal"] > ev["recall_nsigma_equal"]
    assert ev["proposal_cells"] < 0.5 * ev["full_cells"]
