"""GB300 library for BDD-based dual block coordinate ascent on 0-1 ILPs (Lange & Swoboda,
"Efficient Message Passing for 0-1 ILPs with Binary Decision Diagrams").

The compute path is the CUDA library ``_build/libbdd_dbca.so`` behind the C ABI of
``include/bdd_dbca.h``; :mod:`.binding` marshals arguments to it and :class:`Solver` wraps
one instance.
"""
from .binding import (  # noqa: F401
    BDDError, EXPORTED, bdd_bound_parts, bdd_build, bdd_cuthill_mckee, bdd_default_options, bdd_export_canonical, bdd_free,
    bdd_get_state, bdd_iterate, bdd_iterate_device, bdd_iterate_profiled, bdd_last_failed_row, bdd_set_costs,
    bdd_set_state, bdd_sizes, bdd_smooth_backward, bdd_smooth_forward, bdd_strerror, load,
)
from .autograd import smoothed_bound  # noqa: F401
from .solver import Solver, cuthill_mckee  # noqa: F401
