"""Test configuration: registers the ``gpu`` marker.

Tests marked ``gpu`` need a CUDA device and the built library; everything
else runs on the CPU (the oracle's pins, host logic, symbol checks).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a) and the built libsemr")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def _build_native():
    """Compile the oracle (gcc) and libsemr (nvcc, sm_103a) if stale, so that
    test modules can import them.  Both builds are plain compiles."""
    import importlib.util

    import oracle
    oracle.build()
    # load the build script by path: importing the package needs the library
    spec = importlib.util.spec_from_file_location("semr_build", os.path.join(ROOT, "paper_2407_20731_b300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()


_build_native()
