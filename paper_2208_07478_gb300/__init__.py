"""GB300-native periodic CCGF hot path (EOM-IP/EA-CCSD shifted solves + G contraction).

The compute path lives in the C-ABI library built from ``csrc/`` (see
``binding.py``). Importing this package does not load it; ``binding.load()``
does, and raises if it is missing.
"""
