"""GB300-native batched tree-level |M|^2 (arXiv:2507.21039 hot path)."""
