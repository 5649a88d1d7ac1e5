"""GB300-native population fitness scoring for Beagle-style postfix (GCL) programs.

The scoring path is libbeagle.so (CUDA, sm_103a) behind the C ABI in include/beagle.h;
``beagle`` is its Python binding and ``synth`` draws seeded synthetic workloads.
"""
from . import beagle  # noqa: F401
from .beagle import (BeagleError, Dataset, DevicePrograms, score, score_host,  # noqa: F401
                     score_programs, unpack_fitness, upload_dataset, validate_programs)
