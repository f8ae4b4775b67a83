"""GB300-native stage right-hand side of the IB-WENO/TENO method of arXiv:1905.00182."""
