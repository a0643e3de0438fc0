"""GB300-native Monte Carlo radiative transfer (the gCMCRT photon-transport hot path).

Import `paper_2110_15640_gb300.gcmc` for the C-ABI binding; `synth` holds the seeded
synthetic inputs.  Importing the package itself loads nothing.
"""
