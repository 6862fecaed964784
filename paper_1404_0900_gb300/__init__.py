"""GB300-native RR-set engine for TIM / TIM+ influence maximisation.

The compute path lives in the C-ABI library `libtim.so` (hand-written sm_103a CUDA,
see `include/tim.h`); `paper_1404_0900_gb300.tim` is a thin ctypes binding to it and
`paper_1404_0900_gb300.inputs` generates seeded synthetic graphs.
"""
