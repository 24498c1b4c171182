"""GB300-native symmetric Cartesian FMM, standard and angular-momentum-conserving
(arXiv:2107.07166).  The method runs in the CUDA library ``libgbfmm.so`` behind the C ABI
of ``include/gbfmm.h``; ``fmm`` is its Python binding and ``synth`` the seeded input
generators."""
