"""Seeded synthetic inputs (crystal, plane-wave spheres, LDA ground state) shared by the
FP64 oracle and the CUDA path.  Holds no Liouville-Lanczos arithmetic."""
from .cells import (A_LAT, HA_EV, SystemSpec, config_cubic8, config_free_electron, config_kb, config_metal, config_sc16,
                    config_small, config_tiny, config_local_insulator, fft_miller, kmesh_frac, reciprocal, sphere)
from .groundstate import Bundle, build_bundle, bundle_digest, cached_bundle, get_bundle, lda_vxc
