"""GB300-native nonsmooth sphere DEM step for locally refined beds (arXiv 2501.05300)."""
