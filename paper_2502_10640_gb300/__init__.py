"""GB300-native electrostatic PP electron-bunch expansion (arXiv 2502.10640)."""
