"""CPU oracle of arXiv 2204.09131's window MI and searches -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg may
import this package.
"""
