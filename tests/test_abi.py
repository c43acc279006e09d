"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/nbody.h declares (no compute calls here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nbody.h")


def declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import paper_0711_0643_gb300 as pkg
    from paper_0711_0643_gb300 import nbody
    pkg.build()
    return nbody.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_0711_0643_gb300 import nbody
    names = declared()
    assert len(names) >= 25
    out = subprocess.run(["nm", "-D", "--defined-only", nbody.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)
    assert sorted(nbody.EXPORTED) == names


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_0711_0643_gb300 import nbody
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        nbody.load(str(tmp_path / "missing.so"))


def test_config_defaults(lib):
    from paper_0711_0643_gb300 import nbody
    cfg = nbody.nb_config_default()
    assert cfg.eta == 0.01 and cfg.dt_max == 1.0 / 16 and cfg.dt_min == 2.0 ** -40
    assert cfg.precision == nbody.NB_PREC_MIXED and cfg.spin_limit == 1 << 24


def test_build_targets_sm103a_only():
    from paper_0711_0643_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
