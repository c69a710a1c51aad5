"""CPU oracle of the particle-learning cycle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg
may import this package.
"""
