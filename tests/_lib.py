"""Helpers shared by the tests: build-on-demand of libsdx.so and oracle comparisons."""
import os
import threading

_lock = threading.Lock()


def ensure_built():
    from paper_1604_07994_gb300 import build, sdx
    with _lock:
        if not os.path.exists(sdx.LIB_PATH):
            build.build()
    return sdx.load()
