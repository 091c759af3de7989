"""B300-native CNN-preconditioned FGMRES for the 2D Helmholtz equation with PML.

The compute path is the CUDA library `libhelm.so` (sm_103a) behind a C ABI;
`paper_2607_16906_b300.helm` is its thin Python binding.  Importing this
package does not load the library; importing `.helm` does, and fails loudly
when the library is missing.
"""
