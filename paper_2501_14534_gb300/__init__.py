"""GB300 (sm_103a) differentiable Gaussian-splatting rasterizer with the Trick-GS volume and
SH-band masks. The CUDA library is built by ``build.build()``; ``rasterizer`` holds the
torch-facing wrappers (imported lazily, because importing it loads the library)."""
import importlib

__all__ = ["build", "synth", "rasterizer"]


def __getattr__(name):
    if name in ("rasterizer", "build", "synth"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
