"""GB300 (sm_103a) effective block algorithm for the 52 baryon-baryon
four-point correlators of arXiv:1510.00903.

The C ABI is declared in ``include/bbc.h``; ``paper_1510_00903_gb300.bbc``
is its Python binding (a submodule, so that ``paper_1510_00903_gb300.build``
works before the library exists).
"""
