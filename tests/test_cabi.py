"""The C-ABI library loads and exports every symbol include/mhd.h declares (no GPU
needed: nothing is called).  Also checks that the binding's list matches the header."""
import os
import re

from paper_0908_4362_gb300 import build, mhd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"\b(mhd_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    build.build()
    lib = mhd.load_library()
    declared = _declared()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert declared == set(mhd.EXPORTS) | (declared - set(mhd.EXPORTS))
    assert set(mhd.EXPORTS) <= declared


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_0908_4362_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "mhd_oracle" not in txt, f


def test_missing_library_fails_loudly(tmp_path):
    import pytest
    with pytest.raises(ImportError):
        mhd.load_library(str(tmp_path / "nope.so"))


def test_fp32_units_build_without_automatic_contraction():
    """The FP32 sweep bodies are inlined into the single-grid kernels and into the persistent
    batched kernel; both units must be built without automatic FMA contraction (the fusions
    are written out), or the two paths could round differently."""
    from paper_0908_4362_gb300 import build
    flags = dict(build.UNITS)
    for unit in ("kernels_f32.cu", "mhd_batch.cu"):
        assert "--fmad=false" in flags[unit] and "--use_fast_math" not in flags[unit], unit
    assert flags["kernels_f32.cu"] == flags["mhd_batch.cu"]
    assert "--fmad=false" in flags["kernels_f64.cu"]
