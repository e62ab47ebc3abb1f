"""Plain FP64 CPU oracle of the explicit energy-conserving PIC scheme.

Test infrastructure only: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the library.
"""
