"""GB300-native alignment plots (Krusche & Tiskin, arXiv 0909.2000)."""
