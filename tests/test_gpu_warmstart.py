"""What the learned warm start gains: on a 20k-Gaussian thorax scan, after a short plain warm-up, the CNN
(trained on pairs the reconstruction's own forward model renders) proposes every projection's weights;
the proposal must lower the scan loss (else it is rejected and the plain optimisation goes on), and the
warm-started optimisation must then sit below the plain one after the same number of steps."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_cnn_warm_start_beats_plain_optimisation():
    import paper_2506_22280_gb300 as pkg
    from paper_2506_22280_gb300 import digs as D, warmstart as WS
    dev = torch.device("cuda")
    wl = synth.thorax(seed=3, n=20_000)
    gt = wl.extra["gt"]
    f = lambda a: torch.as_tensor(a, dtype=torch.float32, device=dev).contiguous()
    meas = torch.empty(len(wl.views), 256, 256, device=dev)
    for s in range(0, len(wl.views), 128):
        ids = list(range(s, min(s + 128, len(wl.views))))
        pj = pkg.Projector(wl.lattice, [wl.views[i] for i in ids])
        pj.forward(f(gt["mu0"]), f(gt["scale"]), f(gt["quat"]), f(gt["rho"]), f(gt["phi"]), f(gt["w"][ids]),
                   out=meas[s:s + len(ids)])
    lr0 = [0.02, 0.005, 0.002, 0.01, 0.02, 0.01]
    rec = pkg.Reconstruction(wl.mu0, wl.scale, wl.quat, wl.rho, wl.phi, wl.w, wl.lattice,
                             D.adam_config(lr0, [x / 10 for x in lr0], 1000))
    nP, B = len(wl.views), 16
    plan = [[int((s * 7 + j * (nP // B)) % nP) for j in range(B)] for s in range(600)]

    def step(r, s):
        ids = plan[s]
        r.step(meas[torch.as_tensor(ids, device=dev)].contiguous(), ids, [wl.views[i] for i in ids])

    for s in range(100):
        step(rec, s)
    plain, warm = rec.clone(), rec.clone()
    pred = pkg.WeightPredictor(3, seed=0, input_scale=0.25)
    make_views = lambda a: synth.circular_views(a, 1000.0, 1500.0, 256, 256, 1.6, 1.6)
    imgs, cs, W = WS.render_training_pairs(warm, make_views, 4096, pred, seed=1)
    losses = WS.train(pred, imgs, cs, W, epochs=3, batch=256, lr=1e-3)
    assert losses[-1] < 0.7 * losses[0], losses          # the network learns the inverse of the renderer
    res = WS.warm_start(warm, pred, meas, wl.views, np.asarray(wl.angles), list(range(nP)))
    assert res["accepted"] and res["loss_proposal"] < res["loss_plain"], res
    for s in range(100, 186):
        step(plain, s)
        step(warm, s)
    lp = WS.scan_loss(plain, meas, wl.views, plain.w)
    lw = WS.scan_loss(warm, meas, wl.views, warm.w)
    assert plain.status() == 0 and warm.status() == 0
    assert lw < 0.9 * lp, (lw, lp)
