"""GB300-native (sm_103a) stochastic spin-coherent-state trace for radical-pair
recombination yields (Lewis, Fay and Manolopoulos).

* ``paper_1612_09517_gb300.rp``        -- ctypes binding of the C ABI (include/rp.h);
                                          importing it loads ``_lib/librp.so``.
* ``paper_1612_09517_gb300.build``     -- builds ``_lib/librp.so`` for sm_103a.
* ``paper_1612_09517_gb300.workloads`` -- seeded synthetic spin systems.
"""
__version__ = "0.1"
