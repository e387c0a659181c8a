"""FP64 CPU oracle for parametric H- and H^2-matrices (Khan, Chen, Rao, Saibaba).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The library under ``paper_2511_03109_gb300`` never imports it, and it never
imports the library: the two share no code.  Inputs reach both from
``paper_2511_03109_gb300.inputs``, which only draws random numbers.

The oracle is deliberately plain and slow.  It follows the paper step by step
in float64 with NumPy, forming every matrix the paper names explicitly:

* ``cheb``     Chebyshev nodes of the first kind and Lagrange polynomials by
               the product formula (§2.2).
* ``kernels``  the parametric kernel functions (§6, kernel table, plus the
               Gaussian / Matern closed forms of the workloads and two
               polynomial test kernels).
* ``tensor``   little-endian reshapes, mode-2 products, face-splitting and
               Kronecker products (§2.1, App. A.2) and TT-SVD (the compressor of
               Oseledets 2011 that §2.1 names, used in place of TT-cross).
* ``tree``     cluster tree (§3.2, Alg. ConstructClusterTree), admissibility
               (§3.4, App. A.2) and block cluster tree (Alg.
               ConstructBlockClusterTree).
* ``pmatrix``  offline stage (Algs. "Offline Stage: Parametric H-matrix" and
               "... H^2-matrix", §4.4), online stage (Alg. "Online Stage", §4.4;
               App. A.4), MVM for both formats (§4.5, App. A.1) and the dense
               brute-force product K(X, X; theta) X (§1).

Parity status of each function is stated in its module docstring; every
function is pinned by a test in ``tests/test_oracle_*.py``.
"""
