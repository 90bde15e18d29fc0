"""GB300-native renderer for Gabor fields (arXiv 2602.05081).

The compute path is libgf.so (hand-written CUDA for sm_103a behind the C ABI
of include/gf.h); this package is its thin Python binding.  ``_abi`` exposes
every C entry point under the same name; ``api`` adds small conveniences
(building the parameter struct from tensors, a torch.autograd.Function for the
tomography adjoint); ``build`` compiles the library in-tree.  Importing the
binding without a built library raises.
"""
