"""FP64 CPU oracle of the gCMCRT photon-transport path: test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg import this package.
"""
