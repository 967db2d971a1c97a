"""GB300 correction engine for Morse-Smale segmentations under lossy
compression (pMSz, arXiv 2601.01787).

The compute path is libmsz.so (hand-written CUDA for sm_103a behind the C ABI
of include/msz.h); this package only marshals arguments.  ``synth`` makes the
seeded synthetic inputs.  The binding is imported lazily so that ``synth`` can
be used without CUDA.
"""

__all__ = ["directions", "correct", "correct_host", "segment", "compare", "verify", "workspace",
           "workspace_size", "host_workspace_size", "load", "status_str", "MszError", "CorrectResult"]


def __getattr__(name):
    if name in __all__ or name in ("api", "OK", "STUCK", "SELF"):
        import importlib
        api = importlib.import_module(__name__ + ".api")
        return api if name == "api" else getattr(api, name)
    raise AttributeError(name)
