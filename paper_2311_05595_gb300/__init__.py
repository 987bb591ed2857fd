"""GB300 (sm_103a) MG-PCG solver for multiresolution SIMP elasticity
(arXiv 2311.05595): the C ABI lives in libtosolve.so (include/tosolve.h),
`tosolve` is its Python binding."""
