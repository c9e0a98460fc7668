"""GB300-native PtrHash query engine (minimal perfect hashing at HBM throughput)."""
