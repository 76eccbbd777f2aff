"""Plain FP64 CPU oracle for the DFR / complex-step / KIOPS / multistep-EPI method.

TEST INFRASTRUCTURE ONLY.  This package is a slow, literal restatement of the
paper's method (Gaudreault, Charron, Dallerit, Tokman, "High-order numerical
solutions to the shallow-water equations on the rotated cubed-sphere grid",
arXiv 2101.05617) used to check the CUDA path.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with the CUDA library
and never imports the product package.

Modules
-------
geometry        rotated cubed sphere: panel angles (Eq. 81-95), frames (Eq. 59-60),
                metric (Eq. 64-70), Christoffel symbols (Eq. 71-80), interface
                Jacobians (App. C, computed from their geometric definition).
dfr             Gauss-Legendre points, Lagrange basis (Eq. 7-8), extended-node
                flux derivative matrix (Eq. 11-13).
shallow_water   the semi-discrete right-hand side F(q) of Eq. (1)-(2) with the
                AUSM interface flux (App. D/E), in complex arithmetic, and the
                complex-step Jacobian-vector product (Eq. 28).
kiops           phi-function linear combinations (Eq. 29) by adaptive Krylov with
                incomplete orthogonalisation and substepping.
epi             multistep EPI2..6 (Eq. 25, 30, 34-38).
fields          conversion of (h, h_B, Cartesian wind) at nodes into the state q.
testpdes        the semilinear parabolic PDE of Sec. 5.1 (EPI order checks).
"""
