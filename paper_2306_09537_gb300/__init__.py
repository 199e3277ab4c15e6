"""GB300-native QuadSwarm forward-dynamics step (arXiv 2306.09537).

``qs`` is the thin ctypes binding of the C-ABI library ``libquadswarm_gpu.so``
(hand-written sm_103a CUDA); importing it loads the library and fails loudly
when it is missing. ``workloads`` holds the seeded synthetic inputs and loads
no native code.
"""
__all__ = ["qs", "workloads", "QuadSwarmEnv", "RolloutFn"]


def __getattr__(name):
    if name in ("QuadSwarmEnv", "RolloutFn"):
        from . import env as _env
        return getattr(_env, name)
    if name in ("qs", "workloads", "env"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
