"""Failure detection without faulting the GPU.

  - Bounded waits of the staged lattice passes: a test hook makes the
    producer never issue the copies of one batch (nothing is in flight into
    that stage), so the consumers waiting for it run out of their bounded
    wait (set to about a millisecond).  The kernel returns, the host reads
    RBC_ETIMEOUT from rbc_stats, and the context stays usable: a fresh
    solve on the same device afterwards matches the oracle.  Both the
    row-staged pass (periodic box) and the compact pass (tube) are checked.
  - A NaN in one served request's host-side initial state (a cell
    velocity): only that request ends with RBC_EUNSTABLE, the requests
    served beside it in the same packs finish normally.
"""
import numpy as np
import pytest

from oracle import oracle as orc
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


@pytest.mark.parametrize("which", ["staged", "compact"])
def test_starved_wait_times_out_and_the_context_survives(which):
    from paper_1107_4889_gb300.rbc import RBC_ETIMEOUT, RbcError
    if which == "staged":
        geom, cells, params = wl.box_workload(n=32, ncells=8, seed=9)
    else:
        geom = wl.tube(40, 17.0, length=32, body_force=(0.0, 0.0, 4e-6))
        cells, params = None, wl.params()
    s = _solver(geom, cells, params)
    assert s.layout()["compact"] == (which == "compact")
    s.set_wait_limit(2_000_000, starve_batch=3)  # ~1 ms at 2 GHz
    s.step(2)
    with pytest.raises(RbcError) as e:
        s.stats()
    assert e.value.code == RBC_ETIMEOUT
    s.close()
    # the device is still usable: a new solve runs and is right
    g2, c2, p2 = wl.box_workload(n=24, ncells=4, seed=12)
    s2 = _solver(g2, c2, p2)
    s2.step(20)
    f = s2.fields()
    st = s2.stats()
    s2.close()
    o = orc.Oracle(g2, c2, p2)
    o.step(20)
    _, u_o, _ = o.fields()
    o.close()
    assert st["step"] == 20
    assert np.linalg.norm(f["u"] - u_o) <= 1e-5 * np.linalg.norm(u_o)


def test_nan_in_one_served_request_ends_only_that_request():
    from paper_1107_4889_gb300.rbc import RBC_EUNSTABLE, Server
    rng = np.random.default_rng(31)
    reqs = [wl.serving_request(rng, box=(32, 32, 32), walled=w, hematocrit=0.2, rate=3e-4, steps=200,
                               precision="f32") for w in (False, False, True, True)]
    bad = 1
    g, c, p, steps, info = reqs[bad]
    c = dict(c)
    c["vel"] = np.zeros((len(c["pos"]), 3))
    c["vel"][0, 0] = np.nan
    reqs[bad] = (g, c, p, steps, info)
    srv = Server(int(4 * 2 ** 30), max_active=8, tick_steps=20)
    for k, (g, c, p, steps, info) in enumerate(reqs):
        srv.submit(g, c, p, steps, steps // 2, tag=k)
    res = sorted(srv.drain(), key=lambda r: r["tag"])
    srv.close()
    assert [r["tag"] for r in res] == [0, 1, 2, 3]
    for k, r in enumerate(res):
        if k == bad:
            assert r["status"] == RBC_EUNSTABLE, r
        else:
            assert r["status"] == 0 and np.isfinite(r["mean_power"]) and r["steps"] == 200, r
