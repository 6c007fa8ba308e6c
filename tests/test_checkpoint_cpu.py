"""Checkpoints of the learned preconditioner (learn.save_checkpoint / load_checkpoint): host-side
round trips and the refusals that keep a corrupted file away from the preconditioner.  The
parameter count comes from the library's host function sem_mlp_param_count (no GPU needed)."""
import types

import numpy as np
import pytest


@pytest.fixture(scope="module")
def learn():
    from paper_1403_0968_gb300 import build

    build.build()
    from paper_1403_0968_gb300 import learn

    return learn


def _fake_trainer(learn, N, seed):
    n = learn.mlp_param_count(N)
    g = np.random.default_rng(seed)
    return types.SimpleNamespace(N=N, h1=learn.MLP_H1, h2=learn.MLP_H2, m=g.standard_normal(n).astype(np.float32),
                                 v=g.random(n).astype(np.float32), step_count=17, lr=5e-4)


def test_weights_round_trip(learn, tmp_path):
    p = learn.he_init(3, seed=1)
    f = tmp_path / "w.npz"
    learn.save_checkpoint(f, 3, p, jacobi_base=False)
    ck = learn.load_checkpoint(f)
    assert (ck["N"], ck["h1"], ck["h2"], ck["jacobi_base"]) == (3, learn.MLP_H1, learn.MLP_H2, False)
    assert ck["params"].dtype == np.float32 and np.array_equal(ck["params"], p)
    assert "m" not in ck


def test_trainer_state_round_trip(learn, tmp_path):
    p = learn.he_init(2, seed=2)
    tr = _fake_trainer(learn, 2, seed=3)
    f = tmp_path / "t.npz"
    learn.save_checkpoint(f, 2, p, trainer=tr)
    ck = learn.load_checkpoint(f)
    assert np.array_equal(ck["params"], p) and np.array_equal(ck["m"], tr.m) and np.array_equal(ck["v"], tr.v)
    assert ck["step"] == 17 and ck["lr"] == 5e-4 and ck["jacobi_base"]


def test_refusals(learn, tmp_path):
    p = learn.he_init(2, seed=4)
    with pytest.raises(ValueError):  # wrong length for the shape
        learn.save_checkpoint(tmp_path / "a.npz", 3, p)
    with pytest.raises(ValueError):  # a trainer of another shape
        learn.save_checkpoint(tmp_path / "a.npz", 2, p, trainer=_fake_trainer(learn, 3, seed=5))
    # a weight turned NaN after writing: refused on load
    f = tmp_path / "nan.npz"
    learn.save_checkpoint(f, 2, p)
    with np.load(f) as z:
        d = {k: z[k] for k in z.files}
    d["params"] = d["params"].copy()
    d["params"][123] = np.nan
    np.savez(f, **d)
    with pytest.raises(ValueError, match="non-finite"):
        learn.load_checkpoint(f)
    # a truncated parameter vector, another format version, a non-finite moment
    for key, val in (("params", d["params"][:-1]), ("version", np.int64(99))):
        e = dict(d, params=np.nan_to_num(d["params"]))
        e[key] = val
        g = tmp_path / f"bad_{key}.npz"
        np.savez(g, **e)
        with pytest.raises(ValueError):
            learn.load_checkpoint(g)
    tr = _fake_trainer(learn, 2, seed=6)
    tr.v[5] = np.inf
    g = tmp_path / "badv.npz"
    learn.save_checkpoint(g, 2, p, trainer=tr)
    with pytest.raises(ValueError, match="non-finite"):
        learn.load_checkpoint(g)
