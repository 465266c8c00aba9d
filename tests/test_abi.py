"""The C-ABI library loads and exports every entry point include/quark.h declares (CPU only:
no compute call is made), and the product path has no fallback when it is missing."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "quark.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(quark_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("quark_encode_pyramid", "quark_update_fuse", "quark_render_ldm", "quark_create", "quark_load_weights"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2411_16680_b300 import build
    lib_path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (quark_[a-z0-9_]+)", out))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    import ctypes
    L = ctypes.CDLL(lib_path)
    for n in declared_symbols():
        assert hasattr(L, n)


def test_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2411_16680_b300 import quark, synth
    with pytest.raises(quark.QuarkError) as e:
        quark.Context(synth.config_small())
    assert e.value.status == quark.ECUDA


def test_config_validation_on_host():
    from paper_2411_16680_b300 import quark, synth
    bad = [synth.config_small().replace(C=24), synth.config_small().replace(heads=3),
           synth.config_small().replace(scales=[(3, 4)]), synth.config_small().replace(near=5.0, far=1.0),
           synth.QuarkConfig(scales=[(8, 4), (2, 4)])]
    for cfg in bad:
        with pytest.raises(quark.QuarkError) as e:
            quark.Context(cfg)
        assert e.value.status == quark.EINVAL, cfg


def test_missing_library_is_an_error(tmp_path, monkeypatch):
    from paper_2411_16680_b300 import quark
    monkeypatch.setattr(quark, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(quark, "_lib", None)
    with pytest.raises(RuntimeError):
        quark.lib()
