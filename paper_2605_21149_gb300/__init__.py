"""GB300-native (sm_103a) QML power-spectrum and pixel-likelihood library.

Hot path of the QML estimator and the pixel Gaussian likelihood of
arxiv 2605.21149 as hand-written CUDA behind a C ABI (include/qmlgb.h):

    qml_ybuild, qml_synthesize, qml_fisher, qml_estimate, pix_loglike,
    qml_potrf, qml_trsm, qml_gemm

`api` is the thin Python binding (torch tensors or numpy arrays in, same
out).  `synth` draws the seeded synthetic inputs.  Importing the package does
not load the native library; the first API call does, and fails loudly if
libqmlgb.so has not been built (`build.build()`).
"""
__all__ = ["api", "synth", "build"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
