"""The C ABI library loads and exports what include/rgf.h declares; host-only
entry points work without a GPU."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

import workloads

ROOT = Path(__file__).resolve().parents[1]


def declared_symbols():
    text = "\n".join(p.read_text() for p in (ROOT / "include").glob("*.h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rgf_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("rgf_build_ribbon", "rgf_lead_selfenergy", "rgf_conductance", "rgf_conductance_grad"):
        assert s in syms


def test_library_exports_every_declared_symbol(rgflib):
    lib = ctypes.CDLL(str(rgflib._LIB_PATH))
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert set(declared_symbols()) <= set(rgflib.EXPORTS)


def test_status_strings(rgflib):
    for s in range(9):
        assert rgflib.lib.rgf_status_str(s).decode().startswith("RGF_")
    assert rgflib.lib.rgf_version().decode()


@pytest.mark.parametrize("N,L,W,seed,p,eseed", [(11, 7, 0.25, 1, 0.0, 0), (245, 3, 0.1, 5, 0.3, 55),
                                                 (12, 9, 0.4, 2**63 + 5, 0.5, 2**64 - 1)])
def test_c_generator_matches_python_generator(rgflib, N, L, W, seed, p, eseed):
    eps, rem = rgflib.generate_onsite(N, L, -2.7, W, seed, p, eseed)
    assert np.array_equal(eps, workloads.anderson_onsite(N, L, W, seed))
    assert np.array_equal(rem, workloads.edge_removed(N, L, p, eseed))


def test_generator_rejects_bad_sizes(rgflib):
    with pytest.raises(rgflib.RGFError) as e:
        rgflib.generate_onsite(1, 5)
    assert e.value.status == rgflib.RGF_EINVAL
    with pytest.raises(rgflib.RGFError):
        rgflib.generate_onsite(11, 0)


def test_no_oracle_in_product_path():
    # The product package and its CUDA sources never reference the oracle.
    for f in list((ROOT / "paper_1107_5300_gb300").rglob("*.py")) + \
            list((ROOT / "paper_1107_5300_gb300" / "csrc").glob("*")):
        txt = f.read_text(errors="ignore")
        assert "oracle" not in txt.lower(), f
