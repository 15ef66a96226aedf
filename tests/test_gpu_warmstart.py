"""The learned initial guess in the solve (held-out seeds): V-cycles and time
from the plain guess, from the trained network and from an untrained one,
and the fallback to the plain guess when the given guess is unusable
(non-finite or garbage).  The committed weights are trained on seeds
1000-2799; the held-out seeds here are 5000 and up."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1905_08890_gb300 import gr, learn  # noqa: E402

HAVE_WEIGHTS = os.path.exists(learn.WEIGHTS)


@pytest.fixture(scope="module")
def ctx():
    c = gr.Context(learn.N)
    yield c
    c.close()


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))


def test_nan_and_garbage_guesses_fall_back_to_the_plain_guess(ctx):
    src, rho = learn.sources(ctx, 5090)
    ref, rp = learn.solve(ctx, src, rho)
    for bad in ("nan", "garbage"):
        guess = ctx.initial_fields()
        for k, v in guess.items():
            if bad == "nan":
                v.fill_(float("nan"))
            else:
                v.normal_(0.0, 10.0)
        fld, rep = learn.solve(ctx, src, rho, guess=guess, check_guess=1)
        assert rep["status_code"] == gr.GR_OK, rep
        assert all(rep["guess_rejected"]), rep["guess_rejected"]
        assert all(r <= 1e-8 for r in rep["res"])
        for k in gr.FIELDS:
            assert _rel(fld[k], ref[k]) < 1e-6, k


@pytest.mark.skipif(not HAVE_WEIGHTS, reason="no trained weights in the tree")
def test_trained_network_guess_against_plain_and_untrained(ctx):
    net = learn.load(learn.WEIGHTS)
    d = np.load(learn.WEIGHTS)
    untrained = gr.Net(learn.N, seed=123)
    untrained.set_norm(d["in_mean"], d["in_std"], d["out_mean"], d["out_std"])
    seeds = list(learn.TEST_SEEDS)[:4]
    rows = learn.evaluate(ctx, net, seeds, log=None)
    rows_u = learn.evaluate(ctx, untrained, seeds, log=None)
    plain = sum(r["cycles_plain"] for r in rows)
    warm = sum(r["cycles_warm"] for r in rows)
    warm_u = sum(r["cycles_warm"] for r in rows_u)
    print(f"V-cycles over {len(seeds)} held-out solves: plain {plain}, trained guess {warm}, untrained {warm_u}")
    # solutions agree whatever the guess
    assert all(r["max_rel_diff_solutions"] < 1e-6 for r in rows + rows_u)
    # the trained guess never costs cycles; the untrained one is caught by the check
    assert warm <= plain
    assert warm <= warm_u
    assert all(r["rejected"] >= 5 for r in rows_u)
    net.close()
    untrained.close()
