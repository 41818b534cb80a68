"""FP64 CPU oracle for the NIFTy.re metric-vector-product / CG-sampling path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the C-ABI library and its Python binding) never
calls it and has no CPU fallback.

The oracle is a plain, slow, readable restatement of what the method computes,
in float64 numpy, written from the paper (arXiv:2402.16683) and the readings
of it listed per function:

* ``grid``       - harmonic geometry of a regular periodic grid with unit total
                   volume (Sec. "Gaussian Processes", the 128x128 example with
                   ``distances = 1/d``).
* ``dht``        - the Hartley transform used as the "FT" of s = FT o sqrt(P) o xi
                   (Sec. "Gaussian Processes"); numpy.fft serves as the FFT step.
* ``amplitude``  - the non-parametric power-spectrum model sqrt(P)
                   (Sec. "Gaussian Processes", ``add_fluctuations`` parameters),
                   forward, JVP and VJP written out by hand.
* ``cf``         - the correlated field cf(xi) = offset + FT(A * xi) with its JVP
                   and VJP (Sec. "Gaussian Processes", Sec. "Core Components":
                   standardization).
* ``likelihood`` - Fisher weights of the Gaussian and Poisson likelihoods with
                   exponential response (Sec. "Building Up Complex Models",
                   Sec. "Performance": N^-1 is the Poisson Fisher metric).
* ``metric``     - M_p = J^T N^-1 J + 1 applied to tangents and the MGVI
                   right-hand side (Sec. "Performance", Sec. "Variational
                   Inference").
* ``cg``         - textbook conjugate gradients for the linear sample draw
                   (Sec. "Variational Inference", ``draw_linear_kwargs``).
* ``icr``        - iterative charted refinement on a 2-D log-radial chart
                   (Sec. "Gaussian Processes", ICR paragraph).
* ``icr3``       - iterative charted refinement on a 3-D spherical log-radial
                   chart (3x3x3 neighbourhoods, 2x2x2 children).
* ``kl``         - the KL energy of MGVI for fixed residual samples, its
                   gradient, the sample-averaged metric and Newton-CG
                   (Sec. "Variational Inference", the minimiser "M").
* ``geovi``      - the geoVI nonlinear update of a sample residual: Newton
                   iterations on the coordinate equation of the likelihood's
                   standardising transform (Sec. "Variational Inference", "SN").

It shares no code with ``paper_2402_16683_gb300`` and imports nothing from it.
"""
