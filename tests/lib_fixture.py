"""Builds libmgiga.so (host compile, no GPU needed) and imports the binding."""
import functools


@functools.lru_cache(maxsize=1)
def binding():
    from paper_1902_01818_gb300 import build
    build.build()
    from paper_1902_01818_gb300 import mgiga
    return mgiga
