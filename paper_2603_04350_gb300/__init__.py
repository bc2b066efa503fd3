"""GB300-native Exp-ParaDiag (arXiv 2603.04350): hand-written sm_103a CUDA kernels
behind a C ABI (include/expd.h, libexpd.so) with a thin ctypes binding.

    from paper_2603_04350_gb300 import expd
    plan = expd.plan_create(expd.spec_from_problem(problem))
    info = plan.solve_fp(u0, None, U)          # torch CUDA tensors or host arrays

`inputs` holds the seeded synthetic workloads; `build` compiles libexpd.so.
Importing the package loads nothing; the library is opened on first use.
"""
__all__ = ["expd", "inputs", "build"]
__version__ = "1.0.0"
