"""GB300-native exact Euclidean clustering (FEC, arxiv 2208.07678)."""
