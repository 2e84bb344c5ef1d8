"""B300-native differentiable voxelization by the generalized winding number.

* ``dv``       ctypes binding of the C ABI (``include/dv_api.h``, ``libdv.so``)
* ``build``    in-tree nvcc build of ``libdv.so`` for sm_103a
* ``meshgen``  seeded synthetic meshes, grids and upstream gradients
"""
__version__ = "0.1.0"
