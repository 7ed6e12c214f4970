"""bench.py's host-side arithmetic, on CPU: the instruction-issue object beside the HBM
roofline, and the per-field relative L1 differences of the precision workload."""
import numpy as np

import bench


def test_issue_object_counts_only_the_dominant_kind():
    prof = {"fluid_x": (3.0, 2), "fluid_z": (4.0, 2), "fluid_y": (0.0, 0), "ct_x": (9.0, 2)}
    ipc = {"fluid_x": 300.0, "fluid_y": 300.0, "fluid_z": 400.0, "ct_x": 200.0}
    cells = 1_000_000
    d = bench.issue_object("fluid", prof, ipc, cells, 152, 2000.0)
    # (300 x 2 + 400 x 2) x 1e6 instructions in 7 ms
    achieved = (300 * 2 + 400 * 2) * cells / 7e-3 / 1e12
    peak = 152 * 4 * 32 * 2000e6 / 1e12
    assert abs(d["achieved"] - achieved) < 1e-12 and abs(d["peak"] - peak) < 1e-12
    assert abs(d["frac"] - achieved / peak) < 1e-12
    assert set(d["instr_per_cell"]) == {"fluid_x", "fluid_z"}     # no launches of fluid_y


def test_issue_object_absent_without_counts_or_launches():
    assert bench.issue_object("fluid", {"fluid_x": (1.0, 1)}, None, 10, 152, 2070.0) is None
    assert bench.issue_object("fluid", {"ct_x": (1.0, 1)}, {"fluid_x": 1.0}, 10, 152,
                              2070.0) is None


def test_rel_l1_fields_groups_vector_components():
    rng = np.random.default_rng(3)
    b = rng.standard_normal((8, 50))
    b[3] = 0.0                               # a momentum component that vanishes
    a = b.copy()
    a[3] += 1e-3                             # its difference is measured against |m|
    a[0] += 2e-3
    err = bench._rel_l1_fields(a, b)
    den_m = np.abs(b[1:4]).sum()
    assert abs(err[3] - 50e-3 / den_m) < 1e-12
    assert abs(err[0] - 100e-3 / np.abs(b[0]).sum()) < 1e-12
    assert err[5] == err[6] == err[7] == 0.0


def test_ncu_constants_cover_the_current_kernel_sources():
    """The roofline's DRAM traffic and the issue object come from ncu counts keyed by the
    hash of the kernel sources they were taken on; the sources as committed must have them
    (a kernel edit without fresh counts would report traffic as null)."""
    h = bench.kernel_source_hash()
    assert h in bench.NCU_TRAFFIC_PER_CELL, h
    assert h in bench.NCU_INSTR_PER_CELL, h
    ipc = bench.NCU_INSTR_PER_CELL[h]
    assert set(ipc) == {"fluid_x", "fluid_y", "fluid_z", "ct_x", "ct_y", "ct_z"}
    # the fluid sweeps move about their algorithmic bytes per cell
    assert 0.9 * bench.ALG_BYTES["fluid"] <= bench.NCU_TRAFFIC_PER_CELL[h] <= 1.1 * bench.ALG_BYTES["fluid"]
