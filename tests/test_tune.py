"""The schedule autotuner's search and cache (CPU: the timing function is a
stand-in), and one GPU tuning run on a small batch."""
import numpy as np
import pytest

from paper_2604_22625_gb300 import synthetic as S
from paper_2604_22625_gb300 import tune


def _batch():
    return S.config_batch(n_single=24, n_multi=4)


def test_signature_depends_on_shape_not_values():
    a = _batch()
    b = S.config_batch(seed=13, n_single=24, n_multi=4)   # other values, other sizes
    assert tune.signature(a, "bf16", 1e-6) == tune.signature(a, "bf16", 1e-6)
    assert tune.signature(a, "bf16", 1e-6) != tune.signature(a, "f32", 1e-6)
    assert tune.signature(a, "bf16", 1e-6) != tune.signature(a, "bf16", 1e-7)
    assert isinstance(tune.signature(b, "bf16", 1e-6), str)


def test_sample_is_stratified():
    probs = _batch()
    smp = tune.sample(probs, fraction=0.25)
    assert 7 <= len(smp) <= 8
    work = [p.F.shape[0] * max(1, p.T - 1) for p in smp]
    assert work == sorted(work, reverse=True)
    assert max(work) == max(p.F.shape[0] * max(1, p.T - 1) for p in probs)


def test_search_picks_fastest_converging_and_caches(tmp_path):
    probs = _batch()
    calls = []

    def timer(smp, opts):
        calls.append(dict(opts))
        if opts["cta_work"] == 4096.0 and opts["check_every"] == 32:
            return None                                   # did not converge: dropped
        return abs(np.log2(opts["cta_work"] / 8192.0)) + abs(opts["check_every"] - 128) / 100.0 + 1.0

    path = str(tmp_path / "tune.json")
    best = tune.tune(probs, timer=timer, cache_path=path)
    assert (best.cta_work, best.check_every) == (8192.0, 128)
    assert len(calls) == len(tune.CTA_WORK) * len(tune.CHECK_EVERY)
    again = tune.tune(probs, timer=lambda *_: pytest.fail("cached choice must not be re-timed"), cache_path=path)
    assert (again.cta_work, again.check_every) == (8192.0, 128)


@pytest.mark.gpu
def test_gpu_tuning_run(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2604_22625_gb300.build import build
    build()
    probs = [S.make_single(n, 40, 500 + i) for i, n in enumerate([300, 900, 1500, 2200])]
    probs += [S.make_multi(4, 300, 40, 520)]
    best = tune.tune(probs, precision="bf16", tol=1e-6, cache_path=str(tmp_path / "t.json"),
                     cta_work=(2048.0, 8192.0), check_every=(64,), fraction=1.0)
    assert best.seconds > 0 and best.cta_work in (2048.0, 8192.0)
