"""GB300-native approximate max-depth general voting (arXiv 2107.11810)."""
