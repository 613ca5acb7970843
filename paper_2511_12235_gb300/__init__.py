"""Consistent cone-beam system-matrix projectors for GB300 (sm_103a).

Matrix-free forward p = W x and back x = W^T p, where every entry W_ij is the exact
area / volume of voxel j inside the cone of detector element i, evaluated on the fly in
CUDA kernels behind the C ABI of ``include/csm.h``.

The CUDA library is loaded on first use of ``Projector`` (or of the solver / serving
modules); a missing ``_build/libcsm.so`` raises ImportError there: there is no fallback.
"""
__all__ = ["Projector", "ProjectFn"]


def __getattr__(name):
    if name == "Projector":
        from .projector import Projector
        return Projector
    if name == "ProjectFn":
        from .autograd import ProjectFn
        return ProjectFn
    raise AttributeError(name)
