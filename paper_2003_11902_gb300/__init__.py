"""GB300-native MAX-MIN Ant System hot path for the symmetric TSP.

Solution construction (candidate lists, bitmask tabu, weighted reservoir
sampling), tour lengths, iteration/global best with trail limits, and the fused
evaporation/deposit/choice_info pass, as hand-written CUDA for sm_103a behind
the C ABI in include/mmas.h; 2-opt local search; batches of colonies advanced
by shared launches.  ``mmas`` is the Python binding; ``instances``
draws seeded synthetic inputs.
"""
from . import instances
from .mmas import (Batch, Colony, MMASError, Prior, load, mmas_best_tour, mmas_construct, mmas_create,
                   mmas_default_params, mmas_destroy, mmas_get_pheromone, mmas_get_setup,
                   mmas_get_tours, mmas_iterate, mmas_last_error, mmas_set_iteration,
                   mmas_set_pheromone, mmas_stats, mmas_synchronize, mmas_update)

__all__ = ["Batch", "Colony", "MMASError", "Prior", "instances", "load", "mmas_best_tour", "mmas_construct",
           "mmas_create", "mmas_default_params", "mmas_destroy", "mmas_get_pheromone",
           "mmas_get_setup", "mmas_get_tours", "mmas_iterate", "mmas_last_error",
           "mmas_set_iteration", "mmas_set_pheromone", "mmas_stats", "mmas_synchronize",
           "mmas_update"]
