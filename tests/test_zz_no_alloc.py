"""rbc_neighbors_noalloc against rbc_neighbors and the oracle, calls in a row.

Some callers cannot call cudaMalloc -- their device memory is committed to
buffers they do not own, or their host forbids allocation outside its own
pool -- so they cannot lend the workspace rbc_init needs.  For them the
library builds the cell-pair candidate lists with its scratch in a static
device array; the caller passes only the positions and the output buffers.
The lists must equal, bit for bit (the tolerance of every neighbour-list
test), those the time step reports through rbc_neighbors, and the oracle's
brute-force pair list.  Three calls in a row on different boxes -- fully
periodic, walled along y (non-periodic bins clamp at the walls), and a box
only two bins high (2 r_cut < L < 3 r_cut, where the 27-bin scan must not
visit a bin twice) -- check that the shared scratch is cleared between
calls.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1107_4889_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MAXN = 128
RC = wl.PAPER_PARAMS["r_cut"]

# (seed, dims, periodic, cells)
CASES = [
    (41, (48, 48, 48), (1, 1, 1), 400),
    (42, (40, 30, 40), (1, 0, 1), 250),
    (43, (40, 20, 40), (1, 1, 1), 200),
]


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_4889_gb300 import build
    build.build()
    return t


def _geometry(dims, periodic):
    if periodic[1]:
        return wl.periodic_box(*dims)
    return wl.plane_channel(*dims)


def _case(seed, dims, periodic, n):
    rng = np.random.default_rng(seed)
    # walled along y: centres at least 6 from the wall planes (beyond the
    # Gay-Berne range of a wall particle), all three bin rows still used
    lo = np.array([0.0, 0.0 if periodic[1] else 6.0, 0.0])
    hi = np.array(dims, float) - np.array([0.0, 0.0 if periodic[1] else 7.0, 0.0])
    pos = lo + rng.random((n, 3)) * (hi - lo)
    for a in range(3):
        pos[pos[:, a] >= dims[a], a] -= dims[a]
    return pos, wl.random_quaternions(rng, n)


def _step_lists(geom, pos, quat):
    """Lists of the time step (rbc_neighbors after one step of a solver on
    these positions; eps0 = 0: overlapping cells exert no force)."""
    from paper_1107_4889_gb300.rbc import Solver
    s = Solver(geom, wl.cells_dict(pos, quat), wl.params(eps0=0.0, max_neighbors=MAXN, bin_capacity=64))
    s.step(1)
    lists = s.neighbors(MAXN)
    fpos = s.fields(rho=False, u=False)["pos"]
    s.close()
    return lists, fpos


def _oracle_pairs(geom, pos, quat):
    o = orc.Oracle(geom, wl.cells_dict(pos, quat), wl.params(eps0=0.0))
    pairs = {tuple(p) for p in o.neighbor_pairs()}
    o.close()
    return pairs


def test_noalloc_lists_equal_step_lists_and_oracle_calls_in_a_row(torch):
    from paper_1107_4889_gb300 import rbc
    stream = torch.cuda.current_stream().cuda_stream
    refs, outs = [], []
    for seed, dims, per, n in CASES:
        pos, quat = _case(seed, dims, per, n)
        geom = _geometry(dims, per)
        lists, fpos = _step_lists(geom, pos, quat)
        # the step moved nothing (no force, no fluid motion at step 0 beyond
        # rounding); compare on the positions the step's list was built from
        refs.append((lists, _oracle_pairs(geom, fpos, quat), fpos, dims, per, n))
    for lists, pairs, pos, dims, per, n in refs:  # three calls in a row
        pos_d = torch.tensor(pos, dtype=torch.float64, device="cuda")
        counts_d = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        lists_d = torch.full((n, MAXN), -1, dtype=torch.int32, device="cuda")
        rbc.rbc_neighbors_noalloc(pos_d.data_ptr(), n, dims, per, RC, counts_d.data_ptr(), lists_d.data_ptr(),
                                  MAXN, stream)
        outs.append((counts_d.cpu().numpy(), lists_d.cpu().numpy()))
    for (ref, pairs, _, dims, per, n), (counts, lists) in zip(refs, outs):
        assert sum(len(r) for r in ref) > 100
        got = set()
        for i, r in enumerate(ref):
            assert counts[i] == len(r), (dims, i)
            assert np.array_equal(lists[i, : counts[i]], r), (dims, i)
            got |= {(min(i, j), max(i, j)) for j in r}
        assert got == pairs, dims


def test_noalloc_rejects_grids_beyond_the_static_scratch(torch):
    from paper_1107_4889_gb300 import rbc
    # 600^3 box with r_cut 1: 600^3 bins need far more than the 4 MiB scratch
    with pytest.raises(rbc.RbcError) as e:
        rbc.rbc_neighbors_noalloc(0, 0, (600, 600, 600), (1, 1, 1), 1.0, 0, 0, MAXN, None)
    assert e.value.code == rbc.RBC_EINVAL and "static scratch" in str(e.value)
    # a tiny r_cut on an ordinary box: the bin count per axis overflows int
    with pytest.raises(rbc.RbcError) as e:
        rbc.rbc_neighbors_noalloc(0, 0, (64, 64, 64), (0, 0, 0), 1e-12, 0, 0, MAXN, None)
    assert e.value.code == rbc.RBC_EINVAL and "static scratch" in str(e.value)
    # very long axes whose product would wrap a 64-bit count
    with pytest.raises(rbc.RbcError) as e:
        rbc.rbc_neighbors_noalloc(0, 0, (2 ** 30, 2 ** 30, 2 ** 30), (0, 0, 0), 1.0, 0, 0, MAXN, None)
    assert e.value.code == rbc.RBC_EINVAL and "static scratch" in str(e.value)
