"""FP64 CPU oracle for the time-reversible FDTD gradient (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may import this package.  It shares no code with the CUDA path.
"""
