"""GB300-native queue-driven Bellman-Ford SSSP (C-ABI library + thin binding)."""
