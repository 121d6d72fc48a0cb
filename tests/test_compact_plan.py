"""The compact lattice pass's batch table, checked on the host (no GPU).

The set-up packs row segments (a row's fluid range, a fluid run of a
branched row, or a piece of a row) into batches that fill one stage, each
segment with its own sector-aligned window, and precomputes the bulk copies
of each batch with their byte count (the mbarrier's transaction count).  A
mistake there would either drop fluid nodes from the pass, stage outside a
stage, or leave a barrier waiting for bytes that never come; the compiled
checker (tests/compact_plan_check.cu) tests all of it for the tube, a
branched Y, a duct whose rows are wider than a stage, a lattice whose rows
wrap along x, and the four storage / cells combinations."""
import os
import subprocess

import numpy as np
import pytest

from paper_1107_4889_gb300 import build as B
from paper_1107_4889_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    B.build()
    out = str(tmp_path_factory.mktemp("plan") / "compact_plan_check")
    objs = [os.path.join(B.OUT_DIR, f.replace(".cu", ".o")) for f in B.SOURCES if f != "api.cu"]
    cmd = [B.nvcc(), *B.ARCH, "-std=c++17", "-O1", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "compact_plan_check.cu"), *objs, "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


def _duct():
    nx, ny, nz = 300, 20, 20
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:, :, 0] = solid[:, :, nx - 1] = 1
    solid[:, 0, :] = solid[:, ny - 1, :] = 1
    return dict(nx=nx, ny=ny, nz=nz, solid=solid)


def _wrapping():
    geom = wl.plane_channel(17, 19, 23)
    geom["solid"][5:9, 7:10, 6:9] = 1
    return geom


CASES = {
    "tube": lambda: wl.tube(64, 28.0, length=40),
    "ybif": lambda: wl.y_bifurcation(64, 12.0, 8.0),
    "duct": _duct,
    "wrapping": _wrapping,
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("esz,cells", [(4, 1), (4, 0), (2, 1), (2, 0)])
def test_batch_table_covers_every_fluid_node_once(checker, tmp_path, name, esz, cells):
    geom = CASES[name]()
    mask = tmp_path / "mask.bin"
    np.ascontiguousarray(geom["solid"], dtype=np.uint8).tofile(mask)
    r = subprocess.run([checker, str(mask), str(geom["nx"]), str(geom["ny"]), str(geom["nz"]), str(esz), str(cells)],
                       capture_output=True, text=True)
    print(name, esz, cells, r.stdout.strip())
    assert r.returncode == 0, r.stdout
    fields = r.stdout.split()
    assert int(fields[fields.index("fluid") + 1]) == wl.fluid_count(geom)
    # stages are mostly full: the cut segments and packed rows fill them
    # (whole-row FP32 stages without cells leave the rest of a row's stage)
    fill = float(fields[fields.index("fill") + 1])
    assert fill > (0.55 if (esz, cells) == (4, 0) else 0.7), fill
