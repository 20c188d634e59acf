"""GB300-native shifted-system TEM hot path (complex-symmetric multifrontal
LDL^T, multi-RHS solves, residue sums, implicit J.v / J^T.w, LSQR).

The compute path lives in the C-ABI library ``libtem.so`` (CUDA for sm_103a);
``paper_2605_19951_gb300.tem`` is its thin ctypes binding.  Importing this
package does not load the library.
"""
