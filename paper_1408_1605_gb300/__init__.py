"""GB300-native single-GPU BFS (level-synchronous top-down frontier expansion)."""
