"""Oracle for the MF-WQ hot path -- TEST INFRASTRUCTURE, not part of the product.

A plain, slow, float64 CPU statement (numpy / scipy) of what the matrix-free
weighted-quadrature isogeometric k-method computes (Sangalli & Tani,
"Matrix-free weighted quadrature for a computationally efficient isogeometric
k-method").  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA library and its Python binding never import, link or call anything
in this package, and this package imports nothing from them.
"""
from .mfwq_oracle import *  # noqa: F401,F403
