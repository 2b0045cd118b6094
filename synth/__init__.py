"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA library.

This module holds inputs only, none of the configuration-interaction method:

* the single-particle (s.p.) table of a harmonic-oscillator (HO) basis, i.e.
  the list of states (N, l, 2j, 2m) whose occupation bits make up a
  determinant (Sec. 2.1 of the paper: one bit per s.p. state);
* the two-body matrix-element (TBME) tables, drawn from a counter-based
  generator so that any implementation of the same published recipe gets the
  same bits;
* the workload presets (the shapes and sizes of the benchmark problems) and
  the random draws of the batched and served problem mixes;
* the random states of the paper's nonzero-count benchmark (``e1``).

Every function is deterministic in its seed.  Nothing here depends on numpy's
own random streams.
"""

from .sp import ho_sp_table, sp_energies, sp_orbitals
from .tbme import (CH_PP, CH_NN, CH_PN, splitmix64_mix, tbme_gaussian,
                   tbme_tables, tbme_tables_zero)
from .workloads import (PRESETS, Preset, preset, batch_candidates,
                        serve_requests)
from .e1 import E1_RATIO, e1_states

__all__ = [
    "ho_sp_table", "sp_energies", "sp_orbitals",
    "CH_PP", "CH_NN", "CH_PN", "splitmix64_mix", "tbme_gaussian",
    "tbme_tables", "tbme_tables_zero",
    "PRESETS", "Preset", "preset", "batch_candidates", "serve_requests",
    "E1_RATIO", "e1_states",
]
