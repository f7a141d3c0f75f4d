"""FP64 CPU oracle for the FC-Gram Navier-Stokes hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (the CUDA library and its Python binding) never imports, links or
executes anything here, and this package imports nothing from the product.

Every function restates one step of the method of Fontana, Bruno, Mininni and
Dmitruk (FC-Gram pseudospectral Navier-Stokes) in plain float64 NumPy / SciPy,
or in mpmath at 60 digits for the continuation tables, and cites the section
or equation it follows.  Where the paper is silent or inconsistent, the
reading taken is stated in the docstring of the module that takes it
(``fc_tables``: geometry, bandwidth and precision of the fits; ``fc``: grid,
Nyquist treatment and truncation; ``ns``: signs, filter normalisation, stage
steps, pressure units, mean mode, injection and Nusselt definition;
``noise``: the App. A perturbation's mode set, draws and scaling).

Parity status: every function is pinned by a test in ``tests/test_oracle_*``
against closed forms, invariants, brute-force sums or the paper's printed
setups; none is "parity unpinned".
"""
