"""CPU oracle for the loop-cluster update: TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  The product path (paper_1810_07485_gb300) never imports it.
"""
