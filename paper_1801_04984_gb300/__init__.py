"""GB300-native space-time Biot poroelasticity solver (dG(r) in time, Q2/RT1/DGQ1
in space) behind a C ABI (include/biot.h).  The Python binding lives in
`paper_1801_04984_gb300.binding`; importing this package loads nothing."""
