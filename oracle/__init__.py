"""CPU FP64 oracle for the variational-embedding ADMM (Algorithm 6 of arXiv:2106.02682).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference legs, never by the solver package.
"""
