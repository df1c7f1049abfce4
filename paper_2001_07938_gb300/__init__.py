"""GB300 (sm_103a) CSR SpMV library with fused CG and PageRank loops.

The computation is the one the LiLAC compiler offloads to sparse libraries
(Ginsbach, Collie & O'Boyle, "Automatically Harnessing Sparse Acceleration",
CC 2020): y = A x on a device-resident CSR matrix, and the conjugate
gradient and PageRank loops that call it.  The C ABI is include/lilac.h;
``paper_2001_07938_gb300.lilac`` is its Python binding.  Importing this
package loads nothing; the library is loaded on first use.
"""
