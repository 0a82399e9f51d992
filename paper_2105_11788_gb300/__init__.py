"""GB300 (sm_103a) strong-bisimulation partition refinement.

The data-parallel hot path of Martens et al., "A linear parallel algorithm to
compute bisimulation and relational coarsest partitions" (arXiv:2105.11788):
Kanellakis-Smolka style refinement with one splitter per round, marks by one
thread per transition, leader election by concurrent write, as hand-written
CUDA behind the C ABI in include/bisim.h (libbisim.so), with a ctypes binding
(`paper_2105_11788_gb300.bisim`) and seeded LTS generators
(`paper_2105_11788_gb300.lts_gen`).
"""
