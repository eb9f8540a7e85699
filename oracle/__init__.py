"""CPU oracle of the soft-rigid coupled IPC time step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path never does.
"""
