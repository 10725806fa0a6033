"""GB300 (sm_103a) implementation of the Fourier-domain hot path of the t-product toolbox:
tprod, tran, tsvd, tnn, tsn, tubal rank and prox_tnn behind the C ABI of include/tp.h.

Submodules: `tp` (ctypes binding of libtp.so), `build` (nvcc build of libtp.so),
`synth` (seeded synthetic inputs).
"""
