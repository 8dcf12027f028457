"""Plain, slow FP64 CPU oracle of the parity-blocked rotated staggered method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call or link anything here.  The
product library (``paper_2606_03599_gb300``) never imports it and shares no
code with it; both sides receive their inputs from ``workloads``.

Contents:

* ``oracle_apply.c`` -- matrix-free FP64 A_h = B_h C_h B_h^H by neighbour gathers
  (Sec. 3, Eqs. K_def ... discrete_GEP), built into ``_oracle_c.so``.
* ``sparse_ops``     -- the same operators as scipy.sparse matrices, transcribed
  equation by equation (Sec. 3 and 4).
* ``oracle``         -- index maps, block restriction, dense pencils, Fourier
  symbols and closed forms (Sec. 4, 5, App. B, C), the weighted local SVD and the
  reference-medium preconditioner built on it (Sec. 5.4), eigen oracles, merging
  (Sec. 6), Hellmann-Feynman gradients.

Parity status of each function is stated in its docstring; "parity unpinned"
marks a function with no independent pin.
"""
