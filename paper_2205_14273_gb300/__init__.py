"""GB300 (sm_103a) implementation of the data-parallel hot path of
semi-structured algebraic multigrid (Magri, Falgout and Yang, arXiv
2205.14273): SSAMG setup and the V(1,1)-preconditioned CG solve, behind the C
ABI of include/ssamg.h.  ``ssamg`` is the Python binding; ``build_lib``
compiles the CUDA library in-tree."""
