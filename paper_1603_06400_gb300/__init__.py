"""GB300 (sm_103a) forward model and adjoint of fan-beam coded-aperture X-ray
coherent-scatter imaging (Odinaka et al., arXiv:1603.06400), behind the C ABI
of include/caxsi.h.  ``caxsi`` holds the ctypes binding; ``build`` compiles the
CUDA library in-tree."""
