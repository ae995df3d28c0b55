"""FP64 CPU oracle of the Coralai substrate step — TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may import, call or
run anything in this package. The CUDA library and its Python binding never do.
"""
