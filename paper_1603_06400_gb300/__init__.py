"""GB300 (sm_103a) forward model and adjoint of fan-beam coded-aperture X-ray
coherent-scatter imaging (Odinaka et al., arXiv:1603.06400), behind the C ABI
of include/caxsi.h.

Modules: ``caxsi`` (ctypes binding: plans, operators, EM-type and ordered-subset
steps, batches), ``autodiff`` (A, A^T and the update as autograd functions;
unrolled reconstruction), ``warmstart`` (the learned warm start), ``build``
(compiles the CUDA library in-tree)."""
