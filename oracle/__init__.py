"""Oracle: a plain, slow FP64 CPU restatement of the Hadamard-Babich (HB)
volume integrator of arXiv 2210.02698, written from the paper.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` may import or run anything
in this package.  It shares no code with the CUDA path (``paper_2210_02698_gb300``
and its ``csrc``); the one common dependency is the seeded input module
``paper_2210_02698_gb300.workloads``, which holds no arithmetic of the method.

Modules (each function cites the passage it follows):

* ``chebyshev`` - Chebyshev nodes, Lagrange interpolants and the blocked
  interpolation F = T^o F^c T^s (Sec. 4.1, Eq. chebinterp, Eq. chebinterpblock).
* ``tables``    - the tabulated ingredients tau^2, v0, v1 at node pairs
  (Sec. 2, Eq. eikonal, Eq. equVs, Eq. initialv0; Sec. 5.1.1 media).
* ``taylor``    - the near-source Taylor recursions (Sec. 2.2, Eq. recursiveT,
  Eq. recursiveB, Eq. C0, Eq. C1); used to pin ``tables`` and to start
  ``sweep``.
* ``sweep``     - Lax-Friedrichs WENO sweeping for the factored eikonal and
  the transport equations (Sec. 2.3, Eq. faceik, Eq. equVs) on a mesh, for
  media without closed-form ingredients (the Gaussian lens); numerics in
  plain C (``sweep.c``, compiled with gcc on first use).
* ``rays``      - ray tracing of the eikonal and the ray-tube form of the v0
  transport equation (Sec. 2): a mesh-free cross-check of ``sweep``.
* ``inclusion`` - scattering by a curve inclusion (Sec. 3.2): K^{s2s},
  K^{v2s}, K^{s2v} and the total field of Eq. m_v2v_inclu, with the exact
  circle series that pins them.
* ``curve_butterfly`` - K^{s2v} as a single butterfly between the cell tree
  and a K-D tree of the segments (Sec. 4.2, K^{s2v} item): a prototype of
  the compressed surface operators, checked against ``inclusion``.
* ``hb3d``      - the ansatz with d = 3 (half-order f_q), the paper's 3D
  media, closed-form tau, v0, v1 and the exact Green's function of the 3D
  constant-gradient medium (Sec. 5.1.2), the 3D self term (Appendix A.2):
  groundwork for a 3D path.
* ``hankel``    - the Hankel-type functions f_q (Eq. termf).
* ``kernel``    - matrix entries g = v0 f0 + v1 f1 (Eq. babich) and the 2D
  self term (Appendix A, Eq. HankelIntegral2dlemma).
* ``dense``     - the dense sums U = K I and its adjoint (Eq. m_v2v).
* ``cpqr``      - column-pivoted QR interpolative decomposition (Eq. ID).
* ``tree``      - K-D cluster tree and proxy-row rule (Sec. 4.2, Eq. proxyv2v).
* ``butterfly`` - plain HODBF/butterfly construction and apply on small
  grids (Sec. 4.2.1, Eq. transfer_computation ... Eq. butterfly_factors).

Parity status: every function above is pinned by a ``-m "not gpu"`` test
against closed forms, the paper's recursions, library routines used as an
independent definition, or brute force; none is "parity unpinned" except
where a module header says so.
"""
