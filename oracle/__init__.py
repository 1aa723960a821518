"""FP64 CPU oracle for the dispatch map, its implicit gradient and the plan step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or runs
anything here; only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` may.  It shares no code with the CUDA
path: it reads the same plain input dictionaries (drawn by
``paper_2410_13055_gb300.synth``, which holds no method arithmetic) and computes
everything from the paper's definitions written out plainly.

What it follows:

* ``qp``        assembles, for one scenario, the dispatch problem of Eq. 2,
                x*(eta) = argmin c(x) s.t. A(eta) x <= b(eta), for a DC power-flow
                network with generators, curtailable loads, lines with flow and
                angle limits and batteries with state-of-charge dynamics (the
                device mix of Section 3.1), regularised by eps/2 |x|^2 on the
                dispatchable quantities so that the argmin is unique.
* ``ipm``       a Mehrotra predictor-corrector interior-point method on the KKT
                conditions of that QP (the paper solves the same problem with an
                interior-point solver, Section 3).
* ``grad``      the implicit gradient of Section 2.2:
                Delta = gamma + sum_s w_s (d x*_s / d eta)^T grad h_s, by three routes:
                central finite differences, the envelope theorem (h = c only) and
                the implicit function theorem on the active KKT system.
* ``plan``      the projected step eta <- proj_[eta_min, eta_max](eta - alpha Delta).
* ``closed``    independent pins: single-bus water-filling, two-bus line
                congestion, two-hour battery arbitrage, brute-force vertex
                enumeration of tiny LPs.
* ``kkt``       FP64 KKT residuals of any candidate (x, prices).
"""
