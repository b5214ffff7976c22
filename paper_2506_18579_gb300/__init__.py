"""GB300-native (sm_103a) ray-fan tracer for RTM-GD (arXiv 2506.18579)."""
