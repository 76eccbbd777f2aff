"""GB300-native DFR shallow-water hot path: complex-step JVPs inside KIOPS
inside multistep EPI steps (arXiv 2101.05617), behind the C-ABI library
``libswepi.so``.  Importing the package loads nothing; ``swepi`` loads the
library on first use and fails loudly when it is missing."""
