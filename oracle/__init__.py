"""Plain FP64 CPU oracle for the collision operator Q(f,f) and the moment test.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
runs this code; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may call it.  It
shares no code, table or constant generator with the CUDA path: it has its own
quadrature rules, multipliers, transforms (numpy's FFT as a library step),
exponential and fixed-point sums.  Every function cites the passage of
arxiv 2505.03360 (Caparello, Pareschi, Rey) it restates.

Modules
  quadrature  Gauss-Legendre and hemisphere direction rules (sec. 4.4.1, 3D case)
  kernel      Carleman multipliers alpha, alpha', Lambda (sec. 4.4.1, eq. B_F)
  collision   q_fast (FFT sum of convolutions), q_direct (O(N^6) spectral sum)
  classical   classical Fourier-Galerkin kernel B^(l,m) in closed form (eq. Q_k)
  bkw         BKW exact solution for Maxwell molecules (closed-form pin)
  moments     moments, realizability matrices, L1 distance and mask bits
              (sec. 3.2, eq. for V_eps; App. A; sec. 3.3, L1 criterion)
  regime      gradient indicators on the 2D grid (V_eps^1 eigenvalues,
              lambda_B) and the regime update of Algorithm 1 (sec. 3.3, 4.5)
  imex        penalised IMEX steps of df/dt = Q(f)/eps: eq. 1002 and the
              PR(2,2,2) stages (sec. 4.3, 4.4)
  esbgk       ES-BGK Gaussian and operator (sec. 2.2) and its first-order
              IMEX step (sec. 4.3, eq. 1000)
  maxwell2d   fast spectral operator for 2D Maxwell molecules (sec. 4.4.1,
              "The 2d case"), its O(N^4) spectral sum and the 2D BKW solution

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against closed forms, invariants, brute force or an independent formula.
"""
