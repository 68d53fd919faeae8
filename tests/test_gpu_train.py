"""Training of the learned preconditioner behind the C ABI (pic_cnn_train)
and its weights file (pic_cnn_save / pic_cnn_load).

* Training with validation keeps the best scored state, and flexible CG with
  it needs at most half of Jacobi-CG's iterations on a held-out deposit.
* Save, load into a fresh context: the same weights, the same file bytes
  when saved again, the same flexible-CG iteration count.
* Resume: 100 steps, save, load into a fresh context, 100 more steps with
  resume = 1: the Adam step count continues (200), and the resumed run
  starts from the first run's loss level instead of the initial one.
* The smoother target: the V-cycle with the trained smoother needs at most
  one flexible-CG iteration more than with damped Jacobi smoothing.
* Rejected options, resume without weights, corrupted and truncated files.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    import paper_2605_05469_gb300 as pg
    pg.lib()
    return pg


def deposit_rhs(pg, N, seed):
    c = pg.Context().init(N, 8, seed)
    rho = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    c.deposit(rho)
    c.close()
    return rho


def iters(pg, c, rho, pc):
    phi = torch.zeros_like(rho)
    info = c.solve(rho, phi, tol=1e-10, maxit=5000, precision=pg.PREC_MIXED, precond=pc)
    assert info["converged"] and info["rel_res"] <= 1e-10, info
    return info["iters"]


def test_train_save_load_round_trip(pg, tmp_path):
    c = pg.Context().init(128, 0, 0)
    info = c.cnn_train(pg.TRAIN_PRECONDITIONER)
    assert info["steps"] == 600 and 0 <= info["best_step"] <= 600
    assert info["adam_steps"] == info["best_step"] and 0 < info["best_iters"] < 2001
    rho = deposit_rhs(pg, 128, 77)
    it_cnn = iters(pg, c, rho, pg.PC_CNN)
    it_jac = iters(pg, c, rho, pg.PC_JACOBI)
    assert 2 * it_cnn <= it_jac, (it_cnn, it_jac)
    path = str(tmp_path / "w.piccnn")
    c.cnn_save(path)
    assert os.path.getsize(path) == 32 + 3 * 4 * pg.CNN_WEIGHTS
    c2 = pg.Context().init(128, 0, 0)
    c2.cnn_load(path)
    assert np.array_equal(c2.cnn_get_weights(), c.cnn_get_weights())
    path2 = str(tmp_path / "w2.piccnn")
    c2.cnn_save(path2)
    with open(path, "rb") as f1, open(path2, "rb") as f2:
        assert f1.read() == f2.read()
    assert iters(pg, c2, rho, pg.PC_CNN) == it_cnn
    c.close()
    c2.close()


def test_resume_continues_training(pg, tmp_path):
    c = pg.Context().init(64, 0, 0)
    first = c.cnn_train(pg.TRAIN_PRECONDITIONER, steps=100, validate_every=0)
    assert first["adam_steps"] == 100 and first["best_iters"] == -1
    path = str(tmp_path / "r.piccnn")
    c.cnn_save(path)
    c.close()
    c2 = pg.Context().init(64, 0, 0)
    c2.cnn_load(path)
    second = c2.cnn_train(pg.TRAIN_PRECONDITIONER, steps=100, validate_every=0, resume=True)
    assert second["adam_steps"] == 200
    # the resumed run starts where the first one ended, not from the Jacobi start
    assert second["loss_first"] < 0.5 * (first["loss_first"] + first["loss_last"]), (first, second)
    assert second["loss_last"] <= 1.1 * first["loss_last"], (first, second)
    c2.close()


def test_trained_smoother_matches_jacobi_smoothing(pg, capsys):
    c = pg.Context().init(128, 0, 0)
    info = c.cnn_train(pg.TRAIN_SMOOTHER)
    rho = deposit_rhs(pg, 128, 78)
    it_mg = iters(pg, c, rho, pg.PC_MG)
    it_mg_cnn = iters(pg, c, rho, pg.PC_MG_CNN)
    with capsys.disabled():
        print(f"\nmultigrid FCG iterations at 128^3: Jacobi smoothing {it_mg}, trained smoother {it_mg_cnn}; "
              f"training {info}")
    assert it_mg_cnn <= it_mg + 1, (it_mg_cnn, it_mg)
    c.close()


def test_rejects_bad_options_and_files(pg, tmp_path):
    c = pg.Context().init(32, 0, 0)
    for bad in ({"grid": 40}, {"grid": 24}, {"crop": 8}, {"crop": 128}, {"batch": 0}, {"lr": 0.0},
                {"val_grid": 48}, {"target": 7}, {"sets": 0}):
        r = c.cnn_train(**{**{"steps": 1}, **bad}, raise_on_error=False)
        assert r["code"] == pg.PIC_EINVAL, bad
    assert c.cnn_train(steps=1, resume=True, raise_on_error=False)["code"] == pg.PIC_ESTATE
    with pytest.raises(pg.PicError) as e:
        c.cnn_save(str(tmp_path / "none.piccnn"))
    assert e.value.code == pg.PIC_ESTATE
    c.cnn_train(steps=2, validate_every=0)
    path = str(tmp_path / "ok.piccnn")
    c.cnn_save(path)
    raw = open(path, "rb").read()
    for name, data in (("flip", raw[:100] + bytes([raw[100] ^ 1]) + raw[101:]), ("short", raw[:-4]),
                       ("magic", b"XICCNN1\n" + raw[8:]), ("empty", b"")):
        p = str(tmp_path / f"{name}.piccnn")
        with open(p, "wb") as f:
            f.write(data)
        with pytest.raises(pg.PicError) as e:
            c.cnn_load(p)
        assert e.value.code == pg.PIC_EINVAL, name
    with pytest.raises(pg.PicError):
        c.cnn_load(str(tmp_path / "missing.piccnn"))
    c.close()


def test_restarts_keep_the_best_validated_state(pg):
    c = pg.Context().init(64, 0, 0)
    one = c.cnn_train(pg.TRAIN_PRECONDITIONER)
    many = c.cnn_train(pg.TRAIN_PRECONDITIONER, restarts=3)
    assert 0 <= many["best_restart"] < 3
    # restart 0 repeats the plain training (up to the order of FP32 atomics)
    assert many["best_iters"] <= one["best_iters"] + 2, (one, many)
    for bad in ({"restarts": 0}, {"restarts": 17}, {"restarts": 2, "validate_every": 0}):
        assert c.cnn_train(steps=1, raise_on_error=False, **bad)["code"] == pg.PIC_EINVAL, bad
    assert c.cnn_train(steps=1, restarts=2, resume=True, raise_on_error=False)["code"] == pg.PIC_EINVAL
    c.close()
