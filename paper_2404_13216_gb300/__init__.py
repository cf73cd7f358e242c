"""GB300 (sm_103a) BiCGStab / p-BiCGStab with exact dot products (arXiv 2404.13216).

The solver is the C-ABI library ``libpbcg.so`` (include/pbcg.h); ``pbcg`` is
its thin ctypes binding and ``inputs`` the seeded synthetic systems.  Import
``paper_2404_13216_gb300.pbcg`` explicitly: loading it fails loudly when the
library has not been built.
"""
