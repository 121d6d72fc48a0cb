"""Checkpoint and resume (rbc_save / rbc_load).

A run saved at step k and resumed in a fresh handle continues as the
uninterrupted run: bit for bit without cells (the lattice pass has one
writer per value and no atomics), in binary16 with stochastic rounding too
(the checkpoint carries the pass counter that keys the random bits), and
with cells up to the rounding order of the spreading's float atomics (two
uninterrupted runs differ by that much; the bound is 1e-6 relative).  A
checkpoint of another problem is refused.
"""
import numpy as np
import pytest

from paper_1107_4889_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_4889_gb300 import build
    build.build()


def _solver(geom, cells, params):
    from paper_1107_4889_gb300.rbc import Solver
    return Solver(geom, cells, params)


def _split_run(geom, cells, params, k, m):
    """Uninterrupted run of k + m steps, and a run saved at k and resumed
    in a new handle for m more."""
    s = _solver(geom, cells, params)
    s.step(k)
    ck = s.save()
    s.step(m)
    a = s.fields()
    sa = s.stats()
    s.close()
    r = _solver(geom, cells, params)
    r.load(ck)
    r.step(m)
    b = r.fields()
    sb = r.stats()
    r.close()
    assert sa["step"] == sb["step"] == k + m
    return a, b


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_resume_is_bit_identical_without_cells(prec):
    geom = wl.plane_channel(24, 20, 28, body_force=(3e-6, 0.0, 1e-6))
    geom["solid"][8:12, 6:10, 5:9] = 1
    a, b = _split_run(geom, None, wl.params(precision=prec, seed=5), 37, 41)
    assert np.array_equal(a["u"], b["u"]) and np.array_equal(a["rho"], b["rho"])


def test_resume_compact_tube_bit_identical_without_cells():
    geom = wl.tube(40, 17.0, length=24, body_force=(0.0, 0.0, 5e-6))
    a, b = _split_run(geom, None, wl.params(), 30, 31)
    assert np.array_equal(a["u"], b["u"]) and np.array_equal(a["rho"], b["rho"])


def test_resume_with_cells_at_an_odd_step():
    geom, cells, params = wl.box_workload(n=24, ncells=6, body_force=(2e-6, 0, 0), seed=9)
    rng = np.random.default_rng(2)
    cells["vel"] = rng.normal(size=(6, 3)) * 2e-3
    a, b = _split_run(geom, cells, params, 25, 30)
    eu = np.linalg.norm(a["u"] - b["u"]) / np.linalg.norm(a["u"])
    ep = np.abs(a["pos"] - b["pos"]).max()
    print(f"resume with cells: u {eu:.2e}, positions {ep:.2e}")
    assert eu <= 1e-6 and ep <= 1e-8


def test_checkpoint_of_another_problem_is_refused():
    from paper_1107_4889_gb300.rbc import RBC_EINVAL, RbcError
    s = _solver(wl.periodic_box(16), None, wl.params())
    ck = s.save()
    s.close()
    r = _solver(wl.periodic_box(20), None, wl.params())
    with pytest.raises(RbcError) as e:
        r.load(ck)
    assert e.value.code == RBC_EINVAL
    r.close()
