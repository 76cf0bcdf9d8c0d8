"""GB300-native explicit TE/TM wakefield solver (Dohlus & Zagorodnov, Eq. (23)).

The solver itself is the C-ABI library ``libtetm.so`` built from ``csrc/``
(hand-written sm_103a CUDA). ``tetm`` is its thin ctypes binding; importing it
loads the library and fails loudly if it has not been built. ``workloads``
holds the seeded synthetic inputs and imports nothing else from here.
"""

__all__ = ["tetm", "workloads", "sharding"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
