"""GB300-native low-rank NUFFT (Ruiz-Antolin and Townsend, arXiv:1701.04492).

The transform runs in libnufft.so (CUDA kernels for sm_103a behind the C ABI of
include/nufft.h); this package is its thin Python binding:

    from paper_1701_04492_gb300 import Plan, nufft2
    plan = Plan(N, x, eps=1e-9, precision="f32")
    f = plan.forward(c)          # f_j = sum_k c_k exp(-2 pi i x_j k)
    c2 = plan.adjoint(f)         # A^H f

``workloads`` (seeded synthetic inputs) imports without CUDA.
"""

from . import workloads  # noqa: F401


def __getattr__(name):
    # the torch binding is imported on first use, so `workloads` stays light
    if name in ("Plan", "Plan2D", "Batch", "nufft2", "NufftError", "api", "rank", "tune_save", "tune_load",
                "tune_clear"):
        import importlib
        api = importlib.import_module(__name__ + ".api")
        return api if name == "api" else getattr(api, name)
    raise AttributeError(name)
