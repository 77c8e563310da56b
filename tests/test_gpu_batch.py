"""Batched persistent execution of many independent runs (uneven grids and
parameters) against the same runs stepped one at a time, and against the
FP64 oracle."""
import numpy as np
import pytest

from paper_2405_14551_gb300 import workloads as W

from _helpers import CMP_FIELDS, field_errors, make_gpu, make_oracle

pytestmark = pytest.mark.gpu


def small_sweep(seed=11, n=6):
    rng = np.random.default_rng(seed)
    runs = []
    for r in range(n):
        L = int(rng.choice([20, 28, 33, 40]))
        A = float(rng.uniform(0.005, 0.02))
        Ah = float(rng.uniform(0.05, 0.2)) if r % 3 else 0.0
        cen, rad = W.rsa_spheres((L, L, L), 0, rng, 3.0, min(6.0, L / 5), gap=2.0, max_count=int(rng.integers(1, 5)))
        walls = 0b010 if r == 2 else 0
        if walls:
            cen[:, 1] = np.clip(cen[:, 1], 6, L - 7)
        # odd runs use the regularised collision
        p = dict(W.BASE, A_a=A, A_b=A, A_h=Ah, tau_a=0.8 + 0.1 * r, tau_b=1.0, collision=r % 2)
        runs.append(W.Workload(f"run{r}", (L, L + (r % 2), L - 1), walls, p, 100, centres=cen, radii=rad))
    return runs


@pytest.mark.parametrize("storage", ["twoset_f32", "reduced_f16"])
def test_batch_equals_one_at_a_time(storage):
    import paper_2405_14551_gb300.lbcg as L
    runs = small_sweep()
    b = L.Batch(runs, storage=storage)
    tile, bps, ms, cached = b.autotune(steps=2, use_cache=False)
    assert 0 <= tile < L.NUM_TILES and bps in (1, 2, 4) and ms > 0
    b.step(37)  # first step per run, two graph replays, four direct steps
    b.check()
    for r, w in enumerate(runs):
        s = make_gpu(w, storage=storage)
        L.lb_set_tile(s.h, tile)
        s.step(37)
        fb, fs = b.fields(r), s.fields()
        for k in fs:
            np.testing.assert_array_equal(fb[k], fs[k], err_msg=f"run {r} field {k}")


def test_batch_matches_oracle_and_sequential():
    import paper_2405_14551_gb300.lbcg as L
    runs = small_sweep(seed=5, n=4)
    b = L.Batch(runs)
    b.step(5)
    for r in (0, 3):
        o = make_oracle(runs[r])
        o.step(5)
        e = field_errors(b.fields(r), o.fields())
        assert max(e.values()) <= 1e-5, (r, e)
    b2 = L.Batch(runs)
    b2.step_sequential(5)
    for r in range(len(runs)):
        f1, f2 = b.fields(r), b2.fields(r)
        for k in CMP_FIELDS:
            np.testing.assert_array_equal(f1[k], f2[k])


def test_batch_rejects_bad_input():
    import paper_2405_14551_gb300.lbcg as L
    g = [L.make_grid(8, 8, 8), L.make_grid(8, 8, 8)]
    with pytest.raises(L.LBError):
        L.lb_batch_create(g, [L.make_params(storage="twoset_f32"), L.make_params(storage="reduced_f16")])
    with pytest.raises(L.LBError):
        L.lb_batch_create(g, [L.make_params(storage="twoset_f64")] * 2)
    b = L.lb_batch_create(g, [L.make_params()] * 2)
    with pytest.raises(L.LBError):
        L.lb_batch_step(b, 3)  # runs not initialised
    with pytest.raises(L.LBError):
        L.lb_batch_run(b, 2)
    L.lb_batch_destroy(b)
