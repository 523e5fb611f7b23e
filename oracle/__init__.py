"""CPU FP64 oracle for the CSE hot path -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
legs may import this package.  It shares no code with the CUDA path.
"""
