"""GB300-native particle<->mesh field transfer (arXiv 1610.05258)."""
