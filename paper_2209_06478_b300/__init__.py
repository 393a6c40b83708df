"""dynmat on B300: dynamic sparse matrices (COO/CSR/DIA/ELL/HYB switched at run
time), per-format SpMV, format selection and CG, as hand-written sm_103a CUDA
behind the C ABI in include/dynmat.h. `paper_2209_06478_b300.dynmat` is the
Python binding; `paper_2209_06478_b300.build` compiles the library in-tree.
"""
__all__ = ["dynmat", "build"]
