import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")


def pytest_collection_finish(session):
    if session.config.option.collectonly:
        return
    # the oracle runs of the layout parity tests start now, in spawned processes,
    # so that they overlap the GPU tests collected before them
    names = set()
    for item in session.items:
        if item.module.__name__.endswith("test_gpu_layouts"):
            names.update(getattr(item, "callspec", None) and [item.callspec.params.get("name")] or [])
    names.discard(None)
    if names:
        import oracle_pool
        oracle_pool.start(sorted(names))


def pytest_sessionfinish(session, exitstatus):
    if "oracle_pool" in sys.modules:
        sys.modules["oracle_pool"].stop()
