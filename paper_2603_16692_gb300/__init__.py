"""GB300-native CKKS hybrid KeySwitch over RNS (sm_103a CUDA behind a C-ABI).

Importing the package is cheap; the CUDA library is loaded by
``paper_2603_16692_gb300.ks`` on first use.
"""
