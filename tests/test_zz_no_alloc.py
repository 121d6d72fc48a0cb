"""rbc_neighbors_noalloc against rbc_neighbors, two calls in a row.

Some callers cannot call cudaMalloc -- their device memory is committed to
buffers they do not own, or their host forbids allocation outside its own
pool -- so they cannot lend the workspace rbc_init needs.  For them the
library builds the cell-pair candidate lists with its scratch in a static
device array; the caller passes only the positions and the output buffers.
The lists must equal, bit for bit (the tolerance of every neighbour-list
test), those the time step reports through rbc_neighbors.  Two calls in a
row on different boxes check that the shared scratch is cleared between
calls.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_1107_4889_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MAXN = 128


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_4889_gb300 import build
    build.build()
    return t


def _case(seed, L, n):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * L
    pos[pos >= L] -= L
    return pos, wl.random_quaternions(rng, n)


def _reference_lists(pos, quat, L):
    """Lists of the time step: one step of a solver on these positions
    (eps0 = 0: overlapping cells exert no force)."""
    from paper_1107_4889_gb300.rbc import Solver
    s = Solver(wl.periodic_box(L), wl.cells_dict(pos, quat), wl.params(eps0=0.0, max_neighbors=MAXN))
    s.step(1)
    lists = s.neighbors(MAXN)
    s.close()
    return lists


def test_noalloc_lists_equal_step_lists_two_calls_in_a_row(torch):
    from paper_1107_4889_gb300 import rbc
    cases = [(41, 48, 400), (42, 40, 260)]
    data = [_case(*c) for c in cases]
    refs = [_reference_lists(p, q, L) for (p, q), (_, L, _) in zip(data, cases)]
    rc = wl.PAPER_PARAMS["r_cut"]
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for (pos, _), (_, L, n) in zip(data, cases):  # two calls in a row
        pos_d = torch.tensor(pos, dtype=torch.float64, device="cuda")
        counts_d = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        lists_d = torch.full((n, MAXN), -1, dtype=torch.int32, device="cuda")
        rbc.rbc_neighbors_noalloc(pos_d.data_ptr(), n, (L, L, L), (1, 1, 1), rc, counts_d.data_ptr(),
                                  lists_d.data_ptr(), MAXN, stream)
        outs.append((counts_d.cpu().numpy(), lists_d.cpu().numpy()))
    for ref, (counts, lists) in zip(refs, outs):
        assert sum(len(r) for r in ref) > 100
        for i, r in enumerate(ref):
            assert counts[i] == len(r)
            assert np.array_equal(lists[i, : counts[i]], r)


def test_noalloc_rejects_grids_beyond_the_static_scratch(torch):
    from paper_1107_4889_gb300 import rbc
    # 600^3 box with r_cut 1: 600^3 bins need far more than the 4 MiB scratch
    with pytest.raises(rbc.RbcError) as e:
        rbc.rbc_neighbors_noalloc(0, 0, (600, 600, 600), (1, 1, 1), 1.0, 0, 0, MAXN, None)
    assert e.value.code == rbc.RBC_EINVAL and "static scratch" in str(e.value)
