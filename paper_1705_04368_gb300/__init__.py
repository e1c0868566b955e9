"""GB300-native MD + MDLG hot path (arXiv:1705.04368, Parsa & Wagner).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/mdlg.h``); this package only marshals arguments to it.
"""
from .binding import (MAX_LAGS, MAX_VMAX, POT_LJ_SF, POT_LJ_TS, POT_NONE, SITES_ACCUM, SITES_FIELD,
                      SITES_XI, BatchSimulation, MdlgError, Params, Simulation, bin_snapshots,
                      collision, header_functions, idealgas_bin, lib)

__all__ = ["BatchSimulation", "MAX_LAGS", "MAX_VMAX", "POT_LJ_SF", "POT_LJ_TS", "POT_NONE",
           "SITES_ACCUM", "SITES_FIELD", "SITES_XI", "MdlgError", "Params", "Simulation",
           "bin_snapshots", "collision", "header_functions", "idealgas_bin", "lib"]
