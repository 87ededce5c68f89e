"""GB300-native CSF-amortized interval subdivision (Moroz, arXiv 2406.09857).

The compute path is the C-ABI library ``libvx`` (hand-written CUDA for sm_103a, declared in
``include/vx.h``); :mod:`paper_2406_09857_gb300.vx` is its thin ctypes binding and
:mod:`paper_2406_09857_gb300.synth` draws the seeded synthetic inputs.
"""

__all__ = ["vx", "synth"]


def __getattr__(name):
    if name in __all__:
        import importlib

        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
