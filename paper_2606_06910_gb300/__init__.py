"""GB300-native FDTD + CPML hot path (placeholder; filled in below)."""
