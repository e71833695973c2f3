"""What the trained network gains: a small U-Net trained on the GPU (its own
BF16 tensor-core forward and backward kernels) on SARA solutions of seeded
64 x 64 problems, then held-out problems solved by plain SARA (W = I from
zero and the reweighted passes) and by the learned arm (the prediction and
two reweighted passes), both stopped by the same pass rule without the true
sky. The learned arm needs clearly fewer SDMM iterations."""
import numpy as np
import pytest
import torch

import paper_1502_05037_gb300 as pk
from gpu_util import DEV
from paper_1502_05037_gb300 import warmstart as ws

pytestmark = pytest.mark.gpu


def test_trained_network_cuts_sara_iterations_on_held_out_problems():
    size = ws.Size(64)
    inputs, targets = ws.build_training_set(DEV, size, 128, first_iters=200, pass_iters=120)
    net = pk.Unet(size.n, size.n, 3, 16, max_batch=8, seed=3)
    losses = ws.train(net, inputs, targets, epochs=25, batch=8, lr=2e-3)
    assert losses[-1] < 0.2 * losses[0]
    rows = []
    for s in range(6):
        p = ws.make_problem(ws.EVAL_SEED0 + s, DEV, size)
        ws.start(p, torch.zeros((size.n, size.n), dtype=torch.float32, device=DEV))
        rows.append(ws.compare(p, ws.sara_plain(p, DEV), ws.sara_learned(p, net, DEV)))
        p.plan.close()
    it_plain = np.mean([r["it_plain"] for r in rows])
    it_learned = np.mean([r["it_learned"] for r in rows])
    assert it_learned < 0.8 * it_plain
    # the prediction alone is far better than nothing, the passes from it
    # improve on it and meet the constraints (at this small scale the learned
    # result's SNR stays below the plain one's; the 256 x 256 benchmark
    # measures that quality criterion)
    assert np.mean([r["snr_prediction"] for r in rows]) > 5.0          # x = 0 has 0 dB
    assert np.mean([r["snr_learned"] for r in rows]) > np.mean([r["snr_prediction"] for r in rows]) + 3.0
    assert max(r["ratio_learned"] for r in rows) <= 1 + ws.PASS_EPS_TOL
