"""FP64 CPU oracle of the LB-IB-MLS adhesion step.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may use it; the product path never imports it.
"""
