"""GB300 dense-CRF filtering hot path (arXiv 1608.06192).

Python face of the C ABI in include/dcrf.h.  The entry points keep the C
names (dcrf_lattice_build, dcrf_filter, dcrf_qp_fw, dcrf_dc_cccp,
dcrf_lp_subgrad, dcrf_lp_solve, ...); see ``_abi`` for the marshalling and
``synthetic`` for the seeded workloads.  Nothing here computes on the CPU.
"""

_ABI_NAMES = {
    "dcrf_features", "dcrf_lattice_build", "dcrf_lattice_export", "dcrf_filter", "dcrf_filter_adjoint",
    "dcrf_qp_fw", "dcrf_dc_cccp", "dcrf_lp_subgrad", "dcrf_lp_solve", "dcrf_simplex_project",
    "Lattice", "DcrfError", "lib",
}


def __getattr__(name):
    if name in _ABI_NAMES:
        from . import _abi
        return getattr(_abi, name)
    raise AttributeError(name)
