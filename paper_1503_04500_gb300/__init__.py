"""GB300-native RSAI(tol): residual-based sparse approximate inverse (Jia & Kang).

The package is lazy: importing it loads nothing compiled.  ``rsai`` holds the
Python binding of the C-ABI library ``librsai.so`` (built from ``csrc/``);
``inputs`` holds the seeded synthetic matrix generators.
"""
