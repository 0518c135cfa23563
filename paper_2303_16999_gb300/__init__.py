"""Block-sparse x dense matrix product Y = W.X on GB300 (sm_103a).

W (m x k) holds non-zero b x b blocks, b in {1, 4, 8, 16}; X (k x n) is
dense (Section 3).  The compute runs in hand-written CUDA kernels behind the
C ABI declared in ``include/spmm.h``; ``paper_2303_16999_gb300.spmm`` is a
thin ctypes binding with the same names.  Importing this package does not
load the native library; the first call into ``spmm`` does, and fails loudly
if it has not been built (``python -c "import __graft_entry__ as g; g.build()"``).
"""

__all__ = ["spmm", "workloads"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
