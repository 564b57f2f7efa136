"""CPU oracle for the PDHG hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 NumPy/SciPy code that states what the GPU solver computes,
so that tests can check the GPU results against it.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it;
the product path (``paper_2512_06715_gb300``) never does, and this package
imports nothing from the product either.  Inputs reach it as plain arrays.

Modules
  lp        LP in PDLP form, KKT residuals, objectives, relative KKT error
  scaling   Ruiz (l_inf) then Pock-Chambolle (alpha = 1) diagonal rescaling
  pdhg      PDHG iteration (Sec. II.E) with adaptive steps, restarts and
            termination of Applegate et al. (cited by the paper in Sec. II.E)
  simplex   dense two-phase simplex (Bland's rule) for tiny LPs
  merit     single-bus economic dispatch by merit order (closed form)
  brute     enumeration of commitment schedules on tiny instances
"""
