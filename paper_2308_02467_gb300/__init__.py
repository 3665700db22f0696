"""GB300-native element learning for steady radiative transfer (Du & Stechmann, arXiv 2308.02467).

A thin Python binding of the C ABI in include/elrt.h: every function here only checks and
marshals arguments (torch tensors -> device pointers, the current torch CUDA stream) and calls
the library; all the arithmetic of the method runs in the library's CUDA kernels.  The library
is built in-tree (`paper_2308_02467_gb300.build.build()`); using the binding without it raises
ImportError.  The binding is loaded on first use, so `build` can run before the library exists.
"""

_EXPORTS = (
    "LIB_PATH", "ElrtError", "ANG_FV0", "ANG_DO", "LOCAL_FP64", "LOCAL_FP32_IR", "LOCAL_TF32_IR", "F32", "F64",
    "KRYLOV_F32", "KRYLOV_F16", "PRECOND_NONE", "PRECOND_SWEEP", "LU_PRODUCTS_AUTO", "LU_PRODUCTS_TF32",
    "Disc", "Context", "elrt_lgl", "elrt_phase_matrix", "elrt_node_coords", "elrt_n_nodes", "elrt_n_local",
    "elrt_n_skel", "elrt_n_inflow", "exported_symbols", "elrt_build_local_static", "Net",
    "elrt_build_local_learned", "elrt_solve_batch", "elrt_net_file_info",
)

__all__ = list(_EXPORTS)


def __getattr__(name):
    if name in _EXPORTS:
        from . import _binding
        return getattr(_binding, name)
    raise AttributeError(name)
