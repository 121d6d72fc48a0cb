"""GPU tests of the request server (continuous batching of independent
solves; include/rbc.h, "Request server").

  - a served solve reports the time averages a plain Solver run of the same
    problem gives (work rate sampled after every tick);
  - a solve's result is the same alone and in a mix of requests of other
    sizes that run concurrently (the solves share no memory; the float
    atomics of the spreading make the two differ at rounding level);
  - admission by footprint: an arena that holds only some of the requests
    at once still serves all of them, never over-committing it;
  - binary16 storage (stochastic rounding) reproduces the FP32 effective
    viscosity (time-averaged work rate of the drive) of each solve within
    1 %;
  - invalid and oversized requests are rejected at submit;
  - the packed path against the FP64 oracle: four FP32 solves of different
    sizes, periodic and walled, served together in packs; each one's final
    density and velocity fields and per-cell impulses match the oracle.
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


def _server(arena_gb=8.0, max_active=32, tick=100):
    from paper_1107_4889_gb300.rbc import Server
    return Server(int(arena_gb * 2 ** 30), max_active=max_active, tick_steps=tick)


def _serve(srv, reqs, average_from=0):
    for k, (g, c, p, steps, info) in enumerate(reqs):
        srv.submit(g, c, p, steps, average_from, tag=k)
    res = srv.drain()
    res.sort(key=lambda r: r["tag"])
    assert [r["tag"] for r in res] == list(range(len(reqs)))
    for r in res:
        assert r["status"] == 0, r
    return res


def test_served_solve_matches_plain_solver():
    from paper_1107_4889_gb300.rbc import Solver
    rng = np.random.default_rng(3)
    g, c, p, _, info = wl.serving_request(rng, box=(32, 32, 32), walled=False, hematocrit=0.2, rate=3e-4)
    steps, tick = 400, 100
    srv = _server(tick=tick)
    r = _serve(srv, [(g, c, p, steps, info)], average_from=200)[0]
    srv.close()
    s = Solver(g, c, p)
    powers = []
    for k in range(steps // tick):
        s.step(tick)
        st = s.stats()
        if (k + 1) * tick >= 200:
            powers.append(st["power"])
    s.close()
    assert r["steps"] == steps and r["samples"] == len(powers) == 3
    assert abs(r["mean_power"] / np.mean(powers) - 1.0) < 1e-5, (r["mean_power"], np.mean(powers))


def test_alone_and_in_the_mix():
    rng = np.random.default_rng(11)
    probe = wl.serving_request(rng, box=(48, 48, 48), walled=True, hematocrit=0.3, rate=2e-4, steps=600)
    others = [wl.serving_request(rng, step_scale=0.08) for _ in range(12)]
    srv = _server()
    alone = _serve(srv, [probe], average_from=300)[0]
    mix = _serve(srv, others[:6] + [probe] + others[6:], average_from=300)
    srv.close()
    inmix = mix[6]
    print("alone", alone["mean_power"], "mix", inmix["mean_power"])
    assert inmix["samples"] == alone["samples"]
    assert abs(inmix["mean_power"] / alone["mean_power"] - 1.0) < 1e-4
    # the mix ran concurrently: requests overlapped in time
    spans = sorted((r["t_admit"], r["t_done"]) for r in mix)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))


def test_admission_by_footprint():
    from paper_1107_4889_gb300 import rbc
    rng = np.random.default_rng(5)
    reqs = [wl.serving_request(rng, box=(64, 64, 128), walled=bool(k % 2), steps=200) for k in range(6)]
    need = max(rbc.rbc_workspace_size(g, c, p) for g, c, p, _, _ in reqs)
    srv = _server(arena_gb=2.5 * need / 2 ** 30)  # two at a time
    for k, (g, c, p, steps, _) in enumerate(reqs):
        srv.submit(g, c, p, steps, 0, tag=k)
    peak, res = 0, []
    while True:
        a, q = srv.poll()
        peak = max(peak, a)
        res += srv.results()
        if a == 0 and q == 0:
            break
    res += srv.results()
    srv.close()
    assert 2 <= peak < 6 and len(res) == 6 and all(r["status"] == 0 for r in res)
    # at every admission the solves then running fit in the arena together
    arena = int(2.5 * need)
    for r in res:
        live = [q for q in res if q["t_admit"] <= r["t_admit"] < q["t_done"]]
        assert sum(q["workspace_bytes"] for q in live) <= arena


def test_binary16_serving_viscosity_within_one_percent():
    """Per request, the time-averaged work rate of the drive (inversely
    proportional to the suspension's effective viscosity) with binary16
    storage against the same solve in FP32, over the second half of 3,000
    steps."""
    rng = np.random.default_rng(21)
    base = [wl.serving_request(rng, box=b, walled=w, steps=3000)
            for b, w in (((32, 32, 32), False), ((48, 48, 48), True), ((64, 64, 128), False), ((96, 96, 96), True))]
    srv = _server()
    r16 = _serve(srv, base, average_from=1500)
    r32 = _serve(srv, [(g, c, dict(p, precision="f32"), s, i) for g, c, p, s, i in base], average_from=1500)
    srv.close()
    for a, b, req in zip(r16, r32, base):
        rel = a["mean_power"] / b["mean_power"] - 1.0
        print(req[4], "power f16/f32 - 1 =", rel)
        assert abs(rel) < 1e-2


def test_bad_requests_rejected():
    from paper_1107_4889_gb300.rbc import RbcError, RBC_EINVAL, RBC_ENOMEM
    srv = _server(arena_gb=0.05)
    g, c, p = wl.box_workload()
    with pytest.raises(RbcError) as e:
        srv.submit(g, c, dict(p, tau0=0.3), 10)
    assert e.value.code == RBC_EINVAL
    g2, c2, p2 = wl.channel_workload()
    with pytest.raises(RbcError) as e:
        srv.submit(g2, c2, p2, 10)
    assert e.value.code == RBC_ENOMEM
    srv.close()


def test_served_packs_match_oracle_field_by_field():
    """Four FP32 solves of different box sizes -- two periodic boxes under
    the Kolmogorov drive and two walled channels, hematocrit 0.2 -- served
    at once in ticks of 20 steps.  Each class (periodic, walled) forms a
    pack: one launch per kernel for all its members, the packed lattice pass
    over all their row batches.  The final density and velocity of every
    solve match the FP64 oracle at relative L2 1e-5 (the tolerance of the
    single-solve path), its per-cell hydrodynamic impulse J and velocity at
    1e-5 of their largest value over the cells."""
    from oracle import oracle as orc
    rng = np.random.default_rng(21)
    specs = [((32, 32, 32), False), ((48, 32, 32), False), ((32, 32, 48), True), ((40, 36, 32), True)]
    reqs = [wl.serving_request(rng, box=b, walled=w, hematocrit=0.2, rate=3e-4, steps=80, precision="f32")
            for b, w in specs]
    srv = _server(tick=20)
    for k, (g, c, p, steps, info) in enumerate(reqs):
        srv.submit(g, c, p, steps, 0, tag=k, fields=True)
    res = sorted(srv.drain(), key=lambda r: r["tag"])
    srv.close()
    assert [r["tag"] for r in res] == [0, 1, 2, 3]
    for r, (g, c, p, steps, info) in zip(res, reqs):
        assert r["status"] == 0 and r["steps"] == steps == 80
        o = orc.Oracle(g, c, p)
        o.step(steps)
        rho_o, u_o, _ = o.fields()
        do, co = o.diag(), o.cells()
        o.close()
        f, dg = r["fields"], r["diag"]
        fluid = np.ones(len(rho_o), bool) if g["solid"] is None else g["solid"].reshape(-1) == 0
        eu = np.linalg.norm(f["u"][fluid] - u_o[fluid]) / np.linalg.norm(u_o[fluid])
        er = np.linalg.norm(f["rho"][fluid] - rho_o[fluid]) / np.linalg.norm(rho_o[fluid])
        eJ = np.abs(dg["J"] - do["J"]).max() / np.abs(do["J"]).max()
        eV = np.abs(f["vel"] - co["vel"]).max() / np.abs(co["vel"]).max()
        print(info["box"], "walled" if info["walled"] else "periodic", info["ncells"], "cells:",
              f"u {eu:.2e} rho {er:.2e} J {eJ:.2e} V {eV:.2e}")
        assert eu <= 1e-5 and er <= 1e-5 and eJ <= 1e-5 and eV <= 1e-5
