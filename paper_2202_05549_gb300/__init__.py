"""GB300-native single-GPU engine for annotated kernel launches (after
Lightning, arXiv 2202.05549): annotation-driven chunking, halo pack/unpack,
offset sub-grid execution and spilling to pinned host memory, behind the C
ABI of include/lightning.h.  ``lightning`` is the Python helper."""
from . import _lib  # noqa: F401

__all__ = ["lightning"]
