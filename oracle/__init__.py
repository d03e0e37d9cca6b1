"""CPU oracle of the PMWA sweep and exact diagonalisation.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline / reference leg of bench.py.  The GPU product path never imports
it and shares no code with it.
"""
