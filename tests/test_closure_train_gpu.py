"""What the trained closure gains over the method without it.

Coupled runs of the small clustered bed (1x1x0.5 box, fine 128x128x64,
ratio 4, 500,000 log-normal spheres in 200 clusters, Di Felice, gravity,
dt 1e-4) with the fluid relaxed by the coupling source each step.  The
closure is trained on the GPU (cg_mlp_features, cg_mlp_train_step) from
seeds 0 and 1 with the bulk record refreshed every 2, 5 and 10 steps, and
scored on held-out seed 2 against the plain path with a fresh average on
every step: the relative L2 drag error of the learned drag must be well
below that of the stale drag (c = 1) at every refresh interval, with few
rows falling back, for either activation of the closure.
"""
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pairs(cuda_lib):
    from paper_1807_11834_gb300 import closure
    F, T = closure.generate_pairs(synth.small_clustered_bed, seeds=(0, 1), refreshes=(2, 5, 10), steps=12,
                                  n_pairs=400_000)
    assert F.shape[0] >= 390_000 and T.shape == (F.shape[0],)
    return F, T


@pytest.fixture(scope="module", params=["gelu", "relu"])
def trained(pairs, request):
    from paper_1807_11834_gb300 import closure
    F, T = pairs
    m, hist = closure.train(F, T, epochs=20, batch=16384, lr=2e-3, activation=request.param)
    print(request.param, "loss (standardised)", hist[0], "->", hist[-1])
    assert m.activation == request.param
    assert hist[-1] < 0.2 * hist[0]
    yield closure, m
    m.close()


@pytest.mark.parametrize("refresh", [2, 5, 10])
def test_learned_drag_beats_stale_drag(trained, refresh):
    closure, m = trained
    r = closure.evaluate(m, synth.small_clustered_bed, seed=2, refresh=refresh, steps=12)
    print("refresh", refresh, r)
    assert r["err_stale"] > 0          # the fluid did evolve between refreshes
    assert r["err_learned"] < 0.25 * r["err_stale"]
    assert r["fallback_share"] < 0.01


def test_stale_error_grows_with_record_age(trained):
    closure, m = trained
    e = [closure.evaluate(m, synth.small_clustered_bed, seed=2, refresh=k, steps=12)["err_stale"] for k in (2, 10)]
    assert e[1] > 2 * e[0]
