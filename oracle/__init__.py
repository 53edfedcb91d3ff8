"""FP64 CPU oracle of the DPM hot path.

Test infrastructure only: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py.  The product package never imports it.
"""
