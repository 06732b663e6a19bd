"""GB300-native relativistic lattice Boltzmann step with a quasiparticle EOS
(Romatschke, arXiv:1108.5561): C-ABI CUDA library plus a thin Python front end."""
from ._lib import (RLB_BF16, RLB_EOS_CONFORMAL, RLB_EOS_CONST_MASS, RLB_EOS_CROSSOVER, RLB_F32,
                   RLB_F64, RLB_MILNE, RLB_MINKOWSKI, RLB_RADIAL_LAGUERRE, RLB_RADIAL_PAPER,
                   RLBError)
from .run import HBARC, Z_QCD, EosParams, Event, GridParams, Run, alu_peaks, wait_selftest

__all__ = ["Run", "alu_peaks", "wait_selftest", "Event", "GridParams", "EosParams", "RLBError", "HBARC", "Z_QCD", "RLB_F64", "RLB_F32",
           "RLB_BF16", "RLB_EOS_CROSSOVER", "RLB_EOS_CONST_MASS", "RLB_EOS_CONFORMAL",
           "RLB_RADIAL_PAPER", "RLB_RADIAL_LAGUERRE", "RLB_MILNE", "RLB_MINKOWSKI"]
