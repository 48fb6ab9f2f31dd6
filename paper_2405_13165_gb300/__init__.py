"""GB300-native per-particle operator pipeline of the meshfree 3D/2D
model-adaptive flow method (Suchde, arXiv 2405.13165).

Modules: ``mafp`` (ctypes binding of libmafp.so, the C ABI of include/mafp.h),
``pipeline`` (device buffers and the call sequence of one pass), ``autograd``
(torch.autograd.Function over the forward and backward kernels), ``clouds``
(seeded synthetic inputs), ``build`` (nvcc build of libmafp.so for sm_103a).
"""
