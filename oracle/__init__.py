"""CPU oracle of the gCTD transport (TEST INFRASTRUCTURE).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  The product library never does.
"""
