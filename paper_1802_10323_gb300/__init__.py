"""GB300-native eigenfunction-expansion Poisson solver (Costa 2018, §2.1).

``binding`` loads the CUDA C-ABI library (``libps_poisson.so``) and raises if it
is missing; ``synth`` holds the seeded input generators and does not need the
library.
"""
